"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Element-by-element comparisons on seeded inputs at sizes the oracle finishes
in seconds (several tiles of every kernel plus ragged tails), and at the
benchmark's full sizes on sampled outputs that the oracle computes one by
one.  Edge cases: empty slices and empty K, a single event, every event on
one pixel, events on the sensor border, sensors smaller than the window,
zero window radii, out-of-range events and indices.
"""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import (EMB_TOL_FP32, FLOW_FLOOR, FLOW_TOL, emb_rel_err, flow_rel_err, make,
                          to_dev, within_half_bound)


def _check_flow(flow, emb_ref, w, mode):
    ref = oracle.mlp(emb_ref, w.W1, w.b1, w.W2, w.b2)
    if mode == vk.MLP_FP32:
        err = flow_rel_err(flow, ref, FLOW_FLOOR)
        assert err.max() <= FLOW_TOL[mode], (err.max(), err.mean())
    else:
        r = within_half_bound(flow, ref, emb_ref, w, mode)
        assert r <= 1.0, r

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _oracle_emb(sl, D, dx, dy, dt, TXY, K=None):
    T, X, Y = TXY
    return oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, dx, dy,
                                float(dt), T, X, Y, K=K)[0]


CASES = [
    # W, H, n, span_us, D, dx, dy, dt_us
    (346, 260, 20_000, 10_000, 64, 10, 10, 16_000),   # the 346x260 workload, full size
    (97, 61, 3_000, 30_000, 64, 10, 10, 16_000),       # ragged sensor
    (200, 150, 8_000, 50_000, 128, 8, 8, 12_000),      # D=128, 17x17 window
    (64, 40, 2_500, 20_000, 64, 3, 7, 16_000),         # dx != dy
    (45, 33, 1_500, 5_000, 192, 0, 2, 16_000),         # dx = 0, D=192
    (15, 9, 600, 10_000, 256, 10, 10, 16_000),         # sensor smaller than the window, D=256
    (120, 90, 5_000, 20_000, 64, 20, 18, 16_000),      # window wider than 32: a cleared sum grid
]


@pytest.mark.parametrize("W,H,n,span,D,dx,dy,dt", CASES)
def test_encode_matches_oracle(W, H, n, span, D, dx, dy, dt):
    sl = synth.event_slice(W, H, n, span, n_edges=6, frac_noise=0.1, seed=W * 7 + n)
    enc, TXY, _ = make(sl, D, dx, dy, dt)
    x, y, t = to_dev(sl)
    emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    enc.sync_status()
    ref = _oracle_emb(sl, D, dx, dy, dt, TXY)
    err = emb_rel_err(emb, ref)
    assert err.max() <= EMB_TOL_FP32, (err.max(), np.argmax(err))


def test_encode_matches_adjacency_form():
    sl, D = synth.workload("slice-346x260-20k")
    enc, TXY, _ = make(sl, D)
    x, y, t = to_dev(sl)
    K = np.random.default_rng(0).choice(sl.n, 400, replace=False).astype(np.int64)
    emb = enc.encode(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    T, X, Y = TXY
    ref, _ = oracle.encode_direct(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                  16_000.0, T, X, Y, K=K)
    assert emb_rel_err(emb, ref).max() <= EMB_TOL_FP32


def test_subset_K_with_repeats_equals_rows_of_full():
    sl = synth.event_slice(120, 90, 5_000, 20_000, seed=5)
    enc, TXY, _ = make(sl, 64)
    x, y, t = to_dev(sl)
    K = np.array([4999, 0, 17, 17, 2500, 3, 3, 3], np.int64)
    sub = enc.encode(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    ref = _oracle_emb(sl, 64, 10, 10, 16_000, TXY, K=K)
    assert emb_rel_err(sub, ref).max() <= EMB_TOL_FP32
    assert np.array_equal(sub[2], sub[3]) and np.array_equal(sub[5], sub[7])


MODES = [vk.MLP_FP32, vk.MLP_FP16, vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16,
         vk.MLP_BF16 | vk.ACC_FP16]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("W,H,n,D", [(346, 260, 20_000, 64), (150, 100, 6_000, 128),
                                     (90, 70, 333, 64), (60, 40, 97, 128)])
def test_predict_matches_oracle(mode, W, H, n, D):
    sl = synth.event_slice(W, H, n, 10_000, n_edges=8, seed=n + D)
    enc, TXY, w = make(sl, D, mode=mode)
    x, y, t = to_dev(sl)
    flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    enc.sync_status()
    _check_flow(flow, _oracle_emb(sl, D, 10, 10, 16_000, TXY), w, mode)


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_BF16 | vk.ACC_FP16])
def test_explicit_requests_d128(mode):
    """D = 128 with an explicit request list (rows in request order, repeats,
    a ragged last tile): each row equals the full call's row and the oracle."""
    sl = synth.event_slice(200, 150, 12_000, 10_000, n_edges=6, seed=131)
    enc, TXY, w = make(sl, 128, mode=mode)
    x, y, t = to_dev(sl)
    full = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    rng = np.random.default_rng(13)
    K = rng.choice(sl.n, 1_000 + 37, replace=True).astype(np.int64)
    fk = enc.predict(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    enc.sync_status()
    ref = _oracle_emb(sl, 128, 10, 10, 16_000, TXY, K=K)
    _check_flow(fk, ref, w, mode)
    assert np.allclose(fk, full[K], rtol=0, atol=1e-3 * (1 + np.abs(full).max()))


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_FP16 | vk.ACC_FP16])
def test_wide_window_predicts_alternate_cleared_grids(mode):
    # 41 x 37 windows: the row pass reads every pixel, so the pixel sums go
    # to a grid cleared for them (by the previous call's head, else on the
    # side stream); dense and sparse slices alternate on one context.  The
    # column pass normalises blocks of 37 outputs, more than a warp's lanes.
    D, dx, dy = 64, 20, 18
    sls = [synth.event_slice(120, 90, n, 10_000, n_edges=5, seed=600 + i)
           for i, n in enumerate((9_000, 1_500, 9_000, 700))]
    enc, TXY, w = make(sls[0], D, dx, dy, mode=mode, t_span_us=10_000)
    for sl in sls:
        x, y, t = to_dev(sl)
        flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        _check_flow(flow, _oracle_emb(sl, D, dx, dy, 16_000, TXY), w, mode)
    enc.sync_status()


def test_switching_precision_keeps_encoder_state():
    sl = synth.event_slice(100, 80, 4_000, 10_000, seed=77)
    enc, TXY, w = make(sl, 64, mode=vk.MLP_FP32)
    x, y, t = to_dev(sl)
    emb_ref = _oracle_emb(sl, 64, 10, 10, 16_000, TXY)
    for mode in (vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16, vk.MLP_FP16, vk.MLP_FP32):
        enc.set_mlp_mode(mode)
        flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        _check_flow(flow, emb_ref, w, mode)


def test_repeated_calls_clear_accumulators():
    sl = synth.event_slice(80, 60, 3_000, 10_000, seed=9)
    enc, TXY, _ = make(sl, 64)
    x, y, t = to_dev(sl)
    a = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    b = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    assert emb_rel_err(b, a).max() < 1e-6


def test_single_event_and_one_pixel_closed_forms():
    D = 64
    T, X, Y = synth.frequencies(D)
    w = synth.mlp_weights(D)
    p = vk.Params(width=32, height=32, D=D, dt_us=16_000, t_span_us=40_000)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y)
    x = torch.tensor([31], dtype=torch.int16, device="cuda")
    y = torch.tensor([0], dtype=torch.int16, device="cuda")
    t = torch.tensor([123], dtype=torch.int32, device="cuda")
    e = enc.encode(x, y, t, 100).cpu().numpy()
    assert np.max(np.abs(e[0, :D] - 1)) < 1e-6 and np.max(np.abs(e[0, D:])) < 1e-6
    # m events at one pixel: mean of the temporal phases
    ts = np.array([0, 700, 3100, 9000, 39000], np.uint32)
    m = ts.size
    x = torch.full((m,), 7, dtype=torch.int16, device="cuda")
    y = torch.full((m,), 30, dtype=torch.int16, device="cuda")
    e = enc.encode(x, y, torch.from_numpy(ts.view(np.int32)).cuda(), 0).cpu().numpy()
    for k in range(m):
        want = np.mean(np.exp(1j * np.outer((ts.astype(float) - ts[k]) / 16_000.0, T)), axis=0)
        got = e[k, :D] + 1j * e[k, D:]
        assert np.max(np.abs(got - want)) < 2e-6


def test_empty_inputs():
    sl = synth.event_slice(50, 40, 100, 1_000, seed=1)
    enc, _, _ = make(sl, 64)
    z16 = torch.empty(0, dtype=torch.int16, device="cuda")
    z32 = torch.empty(0, dtype=torch.int32, device="cuda")
    out = enc.encode(z16, z16, z32, 0)
    assert out.shape == (0, 128)
    out = enc.predict(z16, z16, z32, 0)
    assert out.shape == (0, 2)
    x, y, t = to_dev(sl)
    out = enc.predict(x, y, t, sl.t_ref, K=torch.empty(0, dtype=torch.int64, device="cuda"))
    assert out.shape == (0, 2)
    enc.sync_status()


def test_oversized_call_is_rejected_before_any_device_work():
    # the size check comes before every other argument check and any launch,
    # so the claimed n never reaches the device
    import ctypes as C
    sl = synth.event_slice(50, 40, 100, 1_000, seed=1)
    enc, _, _ = make(sl, 64)
    x, y, t = to_dev(sl)
    out = torch.empty((4, 2), dtype=torch.float32, device="cuda")
    big = (1 << 30) + 1
    lib = vk.lib()
    for fn in (lib.veckm_encode, lib.veckm_predict, lib.veckm_encode_noalloc):
        st = fn(enc.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                C.c_void_p(t.data_ptr()), big, C.c_uint32(sl.t_ref), None, big,
                C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == vk.VECKM_EINVAL
    assert b"events" in lib.veckm_last_error()
    enc.sync_status()


def test_out_of_range_event_reports_erange_and_skips_it():
    sl = synth.event_slice(60, 50, 2_000, 10_000, seed=3)
    enc, TXY, _ = make(sl, 64, t_span_us=10_000)
    xs = sl.x.copy()
    xs[5] = 60  # off the sensor
    ts = sl.t.copy()
    ts[9] = sl.t_ref + 10_001  # beyond the time span
    xd = torch.from_numpy(xs).cuda()
    yd = torch.from_numpy(sl.y).cuda()
    td = torch.from_numpy(ts.view(np.int32)).cuda()
    emb = enc.encode(xd, yd, td, sl.t_ref).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    enc.sync_status()  # the error word was cleared
    assert np.all(emb[5] == 0) and np.all(emb[9] == 0)
    keep = np.setdiff1d(np.arange(sl.n), [5, 9])
    sub = synth.EventSlice(sl.x[keep], sl.y[keep], sl.t[keep], sl.p[keep], sl.width, sl.height,
                           sl.t_ref)
    ref = _oracle_emb(sub, 64, 10, 10, 16_000, TXY)
    assert emb_rel_err(emb[keep], ref).max() <= EMB_TOL_FP32
    # predictions: pixel-sorted (all events) and indexed (explicit K) paths
    w = synth.mlp_weights(64, 128, 3)
    fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
    for mode in (vk.MLP_FP32, vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16):
        enc.set_mlp_mode(mode)
        for Kd in (None, torch.arange(sl.n, dtype=torch.int64, device="cuda")):
            f = enc.predict(xd, yd, td, sl.t_ref, K=Kd).cpu().numpy()
            with pytest.raises(vk.VeckmError):
                enc.sync_status()
            assert np.all(f[5] == 0) and np.all(f[9] == 0)
            _check_flow(f[keep], ref, w, mode)
    # an event before the slice start
    td2 = td.clone()
    td2[0] = sl.t_ref - 1
    enc.encode(xd, yd, td2, sl.t_ref)
    with pytest.raises(vk.VeckmError):
        enc.sync_status()


def test_index_out_of_range_reports_erange():
    sl = synth.event_slice(60, 50, 500, 10_000, seed=4)
    x, y, t = to_dev(sl)
    for mode in (vk.MLP_FP32, vk.MLP_BF16, vk.MLP_BF16 | vk.ACC_FP16):
        enc, _, _ = make(sl, 64, mode=mode)
        K = torch.tensor([0, 500, -1, 7], dtype=torch.int64, device="cuda")
        f = enc.predict(x, y, t, sl.t_ref, K=K).cpu().numpy()
        with pytest.raises(vk.VeckmError) as ei:
            enc.sync_status()
        assert ei.value.status == vk.VECKM_ERANGE
        assert np.all(f[1] == 0) and np.all(f[2] == 0) and np.any(f[0] != 0)


def test_host_entry_point_matches_device_entry_point():
    sl = synth.event_slice(346, 260, 20_000, 10_000, seed=21)
    emb_ref = None
    for mode in (vk.MLP_FP32, vk.MLP_BF16):
        enc, TXY, w = make(sl, 64, mode=mode)
        if emb_ref is None:
            emb_ref = _oracle_emb(sl, 64, 10, 10, 16_000, TXY)
        x, y, t = to_dev(sl)
        dev = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        hx = torch.from_numpy(sl.x).pin_memory()
        hy = torch.from_numpy(sl.y).pin_memory()
        ht = torch.from_numpy(sl.t.view(np.int32)).pin_memory()
        host = enc.predict_host(hx, hy, ht, sl.t_ref).numpy()
        _check_flow(dev, emb_ref, w, mode)
        _check_flow(host, emb_ref, w, mode)
        K = np.arange(0, sl.n, 7, dtype=np.int64)
        host_k = enc.predict_host(hx, hy, ht, sl.t_ref, K=torch.from_numpy(K)).numpy()
        _check_flow(host_k, emb_ref[K], w, mode)


@pytest.mark.parametrize("mode", [vk.MLP_FP32, vk.MLP_FP16])
def test_stage_timing_records_every_call(mode):
    # With stage timing on, the stages after each timing mark launch in full
    # order instead of chained to the kernel before them: both launch forms
    # give the oracle's flows, in the dense and the direct window form.
    sl = synth.event_slice(100, 80, 4_000, 10_000, seed=2)
    enc, TXY, w = make(sl, 64, mode=mode)
    emb_ref = _oracle_emb(sl, 64, 10, 10, 16_000, TXY)
    x, y, t = to_dev(sl)
    for path in (vk.PATH_DENSE, vk.PATH_DIRECT):
        enc.set_path(path)
        chained = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        enc.set_timing(True)
        for _ in range(3):
            timed = enc.predict(x, y, t, sl.t_ref)
        ms, calls = enc.stage_times()
        enc.set_timing(False)
        assert all(v == 3 for v in calls.values())
        assert all(v >= 0 for v in ms.values())
        assert ms["pool_rows" if path == vk.PATH_DENSE else "gather"] > 0
        assert enc.last_launch_count() >= 4
        if mode == vk.MLP_FP32 or path == vk.PATH_DENSE:  # the direct form's head is FP32
            _check_flow(chained, emb_ref, w, mode)
            _check_flow(timed.cpu().numpy(), emb_ref, w, mode)
        else:
            _check_flow(chained, emb_ref, w, vk.MLP_FP32)
            _check_flow(timed.cpu().numpy(), emb_ref, w, vk.MLP_FP32)
    enc.sync_status()


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_BF16, vk.MLP_FP32, vk.MLP_FP16 | vk.ACC_FP16])
def test_full_size_640x480_sampled(mode):
    """The 640x480, 2M-event workload in the launch configuration the benchmark
    times (MLP_FP16: FP32 pooled grid, FP16 tensor-core head, pooling shapes
    autotuned); the oracle computes a sample of the outputs one by one."""
    sl, D = synth.workload("slice-640x480-2M")
    enc, TXY, w = make(sl, D, mode=mode)
    enc.autotune(sl.width, sl.height)
    x, y, t = to_dev(sl)
    flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    enc.sync_status()
    rng = np.random.default_rng(11)
    K = np.sort(rng.choice(sl.n, 600, replace=False)).astype(np.int64)
    ref = _oracle_emb(sl, D, 10, 10, 16_000, TXY, K=K)
    assert emb_rel_err(emb[K], ref).max() <= EMB_TOL_FP32
    T, X, Y = TXY
    Kd = K[::10]
    refd, _ = oracle.encode_direct(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                   16_000.0, T, X, Y, K=Kd)
    assert emb_rel_err(emb[Kd], refd).max() <= EMB_TOL_FP32
    _check_flow(flow[K], ref, w, mode)


@pytest.mark.parametrize("mode", [vk.MLP_BF16, vk.MLP_BF16 | vk.ACC_FP16, vk.MLP_FP16])
def test_full_size_1280x720_d128_sampled(mode):
    """The 1280x720, 4M-event, D=128 precision workload: FP32 and FP16 storage
    of the pooled grid under a 256 -> 128 -> 2 head on the tensor cores."""
    sl, D = synth.workload("slice-1280x720-4M")
    enc, TXY, w = make(sl, D, mode=mode)
    x, y, t = to_dev(sl)
    flow = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    enc.sync_status()
    K = np.sort(np.random.default_rng(12).choice(sl.n, 300, replace=False)).astype(np.int64)
    ref = _oracle_emb(sl, D, 10, 10, 16_000, TXY, K=K)
    assert emb_rel_err(emb[K], ref).max() <= EMB_TOL_FP32
    _check_flow(flow[K], ref, w, mode)
