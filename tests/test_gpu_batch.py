"""GPU tests of batches: slices of uneven sizes on sensors of different
resolutions encoded in one pass over a canvas, plain and as a captured CUDA
graph plan, against the FP64 oracle on each slice alone and against the
single-slice entry point."""
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

D = 64
SPAN = 20_000


def _ctx(W, H, mode=vk.MLP_FP32, D=D):
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=W, height=H, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=SPAN)
    return vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode), (T, X, Y), w


def _slices(seed, sizes, res):
    out = []
    for i, (n, (W, H)) in enumerate(zip(sizes, res)):
        sl = synth.event_slice(W, H, n, SPAN, n_edges=4, frac_noise=0.1, seed=seed * 100 + i,
                               t0_us=3_000_000 + 1_234_567 * i) if n else \
            synth.EventSlice(np.zeros(0, np.int16), np.zeros(0, np.int16), np.zeros(0, np.uint32),
                             np.zeros(0, np.int8), W, H, 5)
        out.append(sl)
    return out


def _dev(sls):
    keep = []
    for s in sls:
        x, y, t = to_dev(s)
        keep.append(vk.Slice(x, y, t, s.t_ref, s.width, s.height))
    return keep


def _oracle(sl, TXY):
    T, X, Y = TXY
    return oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                16_000.0, T, X, Y)[0]


RES = [(346, 260), (97, 61), (200, 150), (15, 9), (128, 128)]


@pytest.mark.parametrize("mode", [vk.MLP_FP32, vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16])
def test_batch_matches_oracle_per_slice(mode):
    sls = _slices(1, [6_000, 1_500, 0, 300, 4_000], RES)
    enc, TXY, w = _ctx(1024, 1024, mode)
    dsl = _dev(sls)
    flow = enc.predict_batch(dsl).cpu().numpy()
    emb = enc.encode_batch(dsl).cpu().numpy()
    enc.sync_status()
    start = 0
    for s in sls:
        if s.n == 0:
            continue
        ref = _oracle(s, TXY)
        rows = slice(start, start + s.n)
        assert emb_rel_err(emb[rows], ref).max() <= EMB_TOL_FP32
        fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
        if mode == vk.MLP_FP32:
            assert flow_rel_err(flow[rows], fref, FLOW_FLOOR).max() <= FLOW_TOL[mode]
        else:
            assert within_half_bound(flow[rows], fref, ref, w, mode) <= 1.0
        start += s.n
    assert start == flow.shape[0]


def test_batch_equals_single_slice_calls():
    sls = _slices(2, [5_000, 2_000, 800], RES[:3])
    enc, TXY, w = _ctx(800, 600)
    flow = enc.predict_batch(_dev(sls)).cpu().numpy()
    start = 0
    for s in sls:
        single, _, _ = _ctx(s.width, s.height)
        x, y, t = to_dev(s)
        f1 = single.predict(x, y, t, s.t_ref).cpu().numpy()
        d = np.abs(flow[start:start + s.n] - f1).max() / np.abs(f1).max()
        assert d < 1e-5, d
        start += s.n


def test_plan_replays_the_batch_and_picks_up_new_event_values():
    # FP32 head: the plan autotunes its pooling shapes, which reorders FP32
    # sums; in a half-precision mode that can flip the rounding of a product
    sls = _slices(3, [7_000, 3_000, 500, 1_200], RES[:4])
    enc, TXY, w = _ctx(700, 700, vk.MLP_FP32)
    dsl = _dev(sls)
    direct = enc.predict_batch(dsl).cpu().numpy()
    launches = enc.last_launch_count()
    plan = enc.plan(dsl)
    assert plan.kernel_count == launches and launches >= 10
    got = plan.launch().cpu().numpy()
    torch.cuda.synchronize()
    assert np.abs(got - direct).max() <= 1e-5 * np.abs(direct).max()
    # new values in the same buffers: every event moved one pixel right (inside each sensor)
    for s, d in zip(sls, dsl):
        d.x.copy_(torch.from_numpy(np.minimum(s.x + 1, s.width - 1).astype(np.int16)).cuda())
    again = plan.launch().cpu().numpy()
    moved = enc.predict_batch(dsl).cpu().numpy()
    assert np.abs(again - moved).max() <= 1e-5 * np.abs(moved).max()
    assert np.abs(again - direct).max() > 1e-3
    enc.sync_status()
    plan.close()


def test_plan_holds_the_context_buffers():
    sls = _slices(4, [2_000, 1_000], RES[:2])
    enc, TXY, w = _ctx(600, 400, vk.MLP_FP16)
    plan = enc.plan(_dev(sls))
    big = synth.event_slice(346, 260, 20_000, SPAN, seed=9)
    x, y, t = to_dev(big)
    with pytest.raises(vk.VeckmError) as ei:
        enc.predict(x, y, t, big.t_ref)
    assert ei.value.status == vk.VECKM_EBUSY
    with pytest.raises(vk.VeckmError) as ei:
        enc.set_mlp_mode(vk.MLP_BF16)
    assert ei.value.status == vk.VECKM_EBUSY
    plan.launch()
    plan.close()
    enc.predict(x, y, t, big.t_ref)
    enc.set_mlp_mode(vk.MLP_BF16)
    enc.sync_status()


def test_out_of_range_event_in_a_slice_is_reported_and_zeroed():
    sls = _slices(5, [1_000, 1_000], [(64, 48), (80, 40)])
    sls[0].x[7] = 64          # inside the canvas but outside its own 64-wide sensor
    sls[1].t[3] = sls[1].t_ref - 1  # before its slice start
    enc, TXY, w = _ctx(512, 512)
    flow = enc.predict_batch(_dev(sls)).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert np.all(flow[7] == 0) and np.all(flow[1_000 + 3] == 0)
    keep = np.setdiff1d(np.arange(1_000), [7])
    sub = synth.EventSlice(sls[0].x[keep], sls[0].y[keep], sls[0].t[keep], sls[0].p[keep], 64, 48,
                           sls[0].t_ref)
    ref = oracle.mlp(_oracle(sub, TXY), w.W1, w.b1, w.W2, w.b2)
    assert flow_rel_err(flow[keep], ref, FLOW_FLOOR).max() <= 1e-4


def test_one_slice_batch_and_plan_read_the_slice_in_place():
    # one slice is its own canvas: no mapping kernel, the pipeline reads the
    # slice's buffers and applies the same test of sensor and time span
    sls = _slices(8, [6_000], [(346, 260)])
    sls[0].x[11] = 346              # inside the 512-wide context, outside the 346-wide sensor
    sls[0].t[5] = sls[0].t_ref - 1  # before the slice start
    enc, TXY, w = _ctx(512, 512)
    dsl = _dev(sls)
    flow = enc.predict_batch(dsl).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert np.all(flow[11] == 0) and np.all(flow[5] == 0)
    keep = np.setdiff1d(np.arange(6_000), [5, 11])
    sub = synth.EventSlice(sls[0].x[keep], sls[0].y[keep], sls[0].t[keep], sls[0].p[keep], 346,
                           260, sls[0].t_ref)
    ref = oracle.mlp(_oracle(sub, TXY), w.W1, w.b1, w.W2, w.b2)
    assert flow_rel_err(flow[keep], ref, FLOW_FLOOR).max() <= FLOW_TOL[vk.MLP_FP32]
    launches = enc.last_launch_count()
    plan = enc.plan(dsl)
    assert plan.kernel_count == launches
    got = plan.launch().cpu().numpy()
    with pytest.raises(vk.VeckmError):
        enc.sync_status()
    assert np.abs(got - flow).max() <= 1e-5 * np.abs(flow).max()
    # the plan reads the slice's buffers at each launch
    dsl[0].y.copy_(torch.from_numpy(np.minimum(sls[0].y + 1, 259).astype(np.int16)).cuda())
    again = plan.launch().cpu().numpy()
    moved = enc.predict_batch(dsl).cpu().numpy()
    assert np.abs(again - moved).max() <= 1e-5 * np.abs(moved).max()
    assert np.abs(again - flow).max() > 1e-3
    with pytest.raises(vk.VeckmError):
        enc.sync_status()
    plan.close()


def test_batch_that_does_not_fit_the_canvas_is_refused():
    sls = _slices(6, [100] * 6, [(300, 200)] * 6)
    enc, _, _ = _ctx(640, 400)
    with pytest.raises(vk.VeckmError) as ei:
        enc.predict_batch(_dev(sls))
    assert ei.value.status == vk.VECKM_EBUSY
    with pytest.raises(vk.VeckmError) as ei:
        enc.predict_batch(_dev(_slices(6, [100], [(700, 10)])))
    assert ei.value.status == vk.VECKM_EINVAL


def test_empty_batches():
    enc, _, _ = _ctx(1024, 512)
    out = enc.predict_batch([])
    assert out.shape == (0, 2)
    out = enc.predict_batch(_dev(_slices(7, [0, 0], RES[:2])))
    assert out.shape == (0, 2) and enc.last_launch_count() == 0
    plan = enc.plan(_dev(_slices(7, [0], RES[:1])))
    plan.launch()
    assert plan.kernel_count == 0
    plan.close()


def test_autotune_keeps_results_and_returns_valid_shapes():
    sls = _slices(8, [4_000, 2_500, 900], RES[:3])
    enc, TXY, w = _ctx(700, 500, vk.MLP_FP32)
    dsl = _dev(sls)
    before = enc.predict_batch(dsl).cpu().numpy()
    ox, oy, cw, ch = vk.canvas_layout([s.width for s in sls], [s.height for s in sls], 10, 10, 700)
    tuned = enc.autotune(cw, ch)
    assert tuned[0] in (2, 3, 4, 6, 8, 12) and tuned[2] in (2, 3, 4, 6, 8, 12)
    assert 1 <= tuned[1] <= 4 and 1 <= tuned[3] <= 4
    after = enc.predict_batch(dsl).cpu().numpy()
    # FP32 throughout: only the summation order of the pooling may change
    assert np.abs(after - before).max() <= 1e-5 * np.abs(before).max()
    # the FP16 pooled grid has its own tuning entry; after tuning it, results
    # stay within that mode's stated bound of the oracle
    enc.set_mlp_mode(vk.MLP_FP16 | vk.ACC_FP16)
    enc.autotune(cw, ch)
    half = enc.predict_batch(dsl).cpu().numpy()
    start = 0
    for s in sls:
        ref = _oracle(s, TXY)
        fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
        assert within_half_bound(half[start:start + s.n], fref, ref, w,
                                 vk.MLP_FP16 | vk.ACC_FP16) <= 1.0
        start += s.n
    enc.sync_status()
