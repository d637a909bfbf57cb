"""GPU tests of the paper's parameter recipes (Section 2.3: window radii 8 or
10, delta_t 16 or 12 ms at 640x480, D = 64), each autotuned, against the FP64
oracle; and of the Lemma 1 density read-back op against the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import EMB_TOL_FP32, FLOW_FLOOR, FLOW_TOL, emb_rel_err, flow_rel_err, to_dev, \
    within_half_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _enc(r, mode, span):
    T, X, Y = synth.frequencies(r["D"], 0)
    w = synth.mlp_weights(r["D"], 128, 3)
    p = vk.Params(width=r["width"], height=r["height"], D=r["D"], dx=r["dx"], dy=r["dy"],
                  dt_us=r["dt_us"], t_span_us=span)
    return vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode), (T, X, Y), w


@pytest.mark.parametrize("name", sorted(synth.RECIPES))
def test_recipe_matches_oracle_after_autotuning(name):
    r = synth.RECIPES[name]
    span = 2 * r["dt_us"]
    sl = synth.event_slice(r["width"], r["height"], 60_000, span, n_edges=16, n_blobs=4,
                           frac_blobs=0.3, frac_noise=0.05, seed=77)
    x, y, t = to_dev(sl)
    T, X, Y = synth.frequencies(r["D"], 0)
    ref = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, r["D"], r["dx"],
                               r["dy"], float(r["dt_us"]), T, X, Y)[0]
    for mode in (vk.MLP_FP32, vk.MLP_FP16 | vk.ACC_FP16):
        enc, _, w = _enc(r, mode, span)
        tuned = enc.autotune(r["width"], r["height"])
        assert all(v > 0 for v in tuned)
        emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
        assert emb_rel_err(emb, ref).max() <= EMB_TOL_FP32
        flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
        if mode == vk.MLP_FP32:
            # the FP32 bar: every event within 1e-4 relative to
            # max(|flow|, FLOW_FLOOR median |flow|)
            err = flow_rel_err(flow, fref, FLOW_FLOOR)
            assert err.max() <= FLOW_TOL[mode], (err.max(), err.mean())
        else:
            # half operands: the a-priori rounding bound through Eq. 6
            assert within_half_bound(flow, fref, ref, w, mode) <= 1.0
        enc.sync_status()


def test_kde_query_matches_oracle_at_any_integer_offset():
    r = dict(width=200, height=150, D=64, dx=10, dy=10, dt_us=16_000)
    sl = synth.event_slice(200, 150, 4_000, 30_000, n_edges=4, frac_noise=0.1, seed=5)
    enc, (T, X, Y), _ = _enc(r, vk.MLP_FP32, 30_000)
    x, y, t = to_dev(sl)
    emb = enc.encode(x, y, t, sl.t_ref)
    rng = np.random.default_rng(11)
    nq = 3_000
    rows = rng.integers(0, sl.n, nq).astype(np.int64)
    qt = rng.integers(-50_000, 50_000, nq).astype(np.int32)
    qx = rng.integers(-40, 40, nq).astype(np.int32)
    qy = rng.integers(-40, 40, nq).astype(np.int32)
    # the origin, offsets far beyond the slice, and the extremes of int32
    qt[:4] = [0, 2_000_000_000, -2_000_000_000, 2_147_483_647]
    qx[:4] = [0, 30_000, -30_000, -2_147_483_648]
    qy[:4] = [0, -12_345, 12_345, 2_147_483_647]
    dev = lambda a: torch.from_numpy(a).cuda()
    g = enc.kde_query(emb, dev(rows), dev(qt), dev(qx), dev(qy)).cpu().numpy()
    e = emb.cpu().numpy().astype(np.float64)
    want = np.array([oracle.kde_query(e[rows[i]], T, X, Y, qt[i] / 16_000.0, qx[i] / 10.0,
                                      qy[i] / 10.0) for i in range(200)])
    assert np.abs(g[:200] - want).max() < 5e-6
    # the origin reads back the mean real part
    assert abs(g[0] - e[rows[0], :64].mean()) < 1e-6
    enc.sync_status()


def test_kde_query_row_out_of_range_reports_erange():
    r = dict(width=64, height=48, D=64, dx=10, dy=10, dt_us=16_000)
    sl = synth.event_slice(64, 48, 500, 10_000, seed=6)
    enc, _, _ = _enc(r, vk.MLP_FP32, 10_000)
    x, y, t = to_dev(sl)
    emb = enc.encode(x, y, t, sl.t_ref)
    z = torch.zeros(3, dtype=torch.int32, device="cuda")
    rows = torch.tensor([0, 500, -1], dtype=torch.int64, device="cuda")
    g = enc.kde_query(emb, rows, z, z, z).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert g[1] == 0 and g[2] == 0 and g[0] != 0
