"""GPU tests of the direct window form (the per-event window loop of
Algorithm 1) against the FP64 oracle, against the dense pooled form, and of
the switch between them (the runtime model of Eq. runtime)."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import EMB_TOL_FP32, FLOW_FLOOR, FLOW_TOL, emb_rel_err, flow_rel_err, make, \
    to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _ref(sl, D, dx, dy, dt, TXY, K=None):
    T, X, Y = TXY
    return oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, dx, dy,
                                float(dt), T, X, Y, K=K)[0]


CASES = [
    # W, H, n, span, D, dx, dy, dt
    (346, 260, 20_000, 10_000, 64, 10, 10, 16_000),
    (97, 61, 3_000, 30_000, 128, 10, 10, 16_000),
    (64, 40, 2_500, 20_000, 64, 3, 7, 16_000),
    (45, 33, 1_500, 5_000, 192, 0, 2, 16_000),
    (15, 9, 600, 10_000, 256, 10, 10, 16_000),     # sensor smaller than the window
    (300, 40, 1_000, 10_000, 64, 40, 3, 16_000),   # window rows wider than a warp
]


@pytest.mark.parametrize("W,H,n,span,D,dx,dy,dt", CASES)
def test_direct_encode_matches_oracle(W, H, n, span, D, dx, dy, dt):
    sl = synth.event_slice(W, H, n, span, seed=W + n)
    enc, TXY, _ = make(sl, D, dx=dx, dy=dy, dt_us=dt)
    enc.set_path(vk.PATH_DIRECT)
    x, y, t = to_dev(sl)
    emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    assert enc.last_path() == vk.PATH_DIRECT
    ref = _ref(sl, D, dx, dy, dt, TXY)
    assert emb_rel_err(emb, ref).max() <= EMB_TOL_FP32
    enc.sync_status()


@pytest.mark.parametrize("mode", [vk.MLP_FP32, vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16])
def test_direct_predict_matches_oracle_with_subsets_and_repeats(mode):
    sl = synth.event_slice(200, 150, 8_000, 40_000, n_edges=8, frac_noise=0.1, seed=21)
    enc, TXY, w = make(sl, 64, mode=mode)
    enc.set_path(vk.PATH_DIRECT)
    x, y, t = to_dev(sl)
    rng = np.random.default_rng(4)
    K = rng.integers(0, sl.n, 1_500).astype(np.int64)
    K[:10] = K[0]  # repeats
    Kd = torch.from_numpy(K).cuda()
    f = enc.predict(x, y, t, sl.t_ref, K=Kd).cpu().numpy()
    ref = _ref(sl, 64, 10, 10, 16_000, TXY, K=K)
    fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
    # the direct form's perceptron is FP32 whatever the mode
    assert flow_rel_err(f, fref, FLOW_FLOOR).max() <= FLOW_TOL[vk.MLP_FP32]
    fa = enc.predict(x, y, t, sl.t_ref).cpu().numpy()  # all events, in input order
    refa = _ref(sl, 64, 10, 10, 16_000, TXY)
    assert flow_rel_err(fa, oracle.mlp(refa, w.W1, w.b1, w.W2, w.b2), FLOW_FLOOR).max() <= 1e-4
    enc.sync_status()


def test_direct_agrees_with_dense_and_handles_hot_pixels():
    # a third of the events on one pixel: its records span many record chunks
    sl = synth.event_slice(120, 90, 6_000, 20_000, seed=8)
    sl.x[::3] = 60
    sl.y[::3] = 45
    enc, TXY, w = make(sl, 64)
    x, y, t = to_dev(sl)
    enc.set_path(vk.PATH_DENSE)
    dense = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    enc.set_path(vk.PATH_DIRECT)
    direct = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    ref = _ref(sl, 64, 10, 10, 16_000, TXY)
    assert emb_rel_err(direct, ref).max() <= EMB_TOL_FP32
    assert np.abs(direct - dense).max() <= 1e-5
    enc.sync_status()


def test_direct_reports_invalid_indices_and_events():
    sl = synth.event_slice(60, 50, 800, 10_000, seed=3)
    enc, TXY, w = make(sl, 64, t_span_us=10_000)
    enc.set_path(vk.PATH_DIRECT)
    xs = sl.x.copy()
    xs[5] = 60  # off the sensor
    x = torch.from_numpy(xs).cuda()
    _, y, t = to_dev(sl)
    K = torch.tensor([0, 5, 800, -1, 7], dtype=torch.int64, device="cuda")
    f = enc.predict(x, y, t, sl.t_ref, K=K).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert np.all(f[1:4] == 0) and np.any(f[0] != 0) and np.any(f[4] != 0)


def test_auto_switch_follows_the_runtime_model():
    sl, D = synth.workload("slice-640x480-2M", scale=0.1)
    enc, TXY, w = make(sl, D, mode=vk.MLP_FP16 | vk.ACC_FP16)
    x, y, t = to_dev(sl)
    # 500 flows: 441-pixel windows cost ~17 us direct against ~130 us of dense passes
    few = torch.from_numpy(np.arange(0, sl.n, sl.n // 500, dtype=np.int64)[:500]).cuda()
    f_few = enc.predict(x, y, t, sl.t_ref, K=few).cpu().numpy()
    assert enc.last_path() == vk.PATH_DIRECT
    enc.predict(x, y, t, sl.t_ref)
    assert enc.last_path() == vk.PATH_DENSE
    # a model that makes the window loop expensive keeps even few flows dense
    enc.set_path_model(0.43, 1.53, 1e4)
    f_dense = enc.predict(x, y, t, sl.t_ref, K=few).cpu().numpy()
    assert enc.last_path() == vk.PATH_DENSE
    # FP32 direct head vs the FP16 dense head: within the half-precision bar
    K = few.cpu().numpy()
    ref = _ref(sl, D, 10, 10, 16_000, TXY, K=K)
    fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
    assert flow_rel_err(f_few, fref, FLOW_FLOOR).max() <= 1e-4
    enc.sync_status()


def test_direct_path_in_a_batch_plan():
    sls = [synth.event_slice(W, H, n, 20_000, seed=30 + i) for i, (W, H, n) in
           enumerate([(346, 260, 3_000), (97, 61, 800), (200, 150, 1_500)])]
    T, X, Y = synth.frequencies(64, 0)
    w = synth.mlp_weights(64, 128, 3)
    p = vk.Params(width=800, height=600, D=64, t_span_us=20_000)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y)
    enc.set_path(vk.PATH_DIRECT)
    dev = []
    for s in sls:
        xx, yy, tt = to_dev(s)
        dev.append(vk.Slice(xx, yy, tt, s.t_ref, s.width, s.height))
    plan = enc.plan(dev)
    got = plan.launch().cpu().numpy()
    start = 0
    for s in sls:
        ref = _ref(s, 64, 10, 10, 16_000, (T, X, Y))
        fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
        assert flow_rel_err(got[start:start + s.n], fref, FLOW_FLOOR).max() <= 1e-4
        start += s.n
    plan.close()
    enc.sync_status()
