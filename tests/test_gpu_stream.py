"""GPU tests of sliding-window streams: each packet encoded against the
window [t_hi - window, t_hi] matches the FP64 oracle recomputed from scratch
on that window, and the resident fixed-point sums after many packets are bit
identical to sums built from the final window alone (no drift)."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import EMB_TOL_FP32, FLOW_FLOOR, FLOW_TOL, emb_rel_err, flow_rel_err, \
    within_half_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

D = 64
WIN = 32_000  # 2 delta_t


def _enc(W, H, mode=vk.MLP_FP32):
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=W, height=H, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=WIN)
    return vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode), (T, X, Y), w


def _long_stream(W, H, n, span, seed):
    return synth.event_slice(W, H, n, span, n_edges=6, frac_noise=0.1, seed=seed, t0_us=5_000_000)


def _packets(sl, rng, mean_us=3_000):
    """(start index, end index, t_hi) of packets cut at random time boundaries."""
    out = []
    t_end = int(sl.t[-1]) + 1
    t = int(sl.t[0])
    i = 0
    while t < t_end:
        t_hi = t + int(rng.integers(mean_us // 3, 2 * mean_us))
        j = int(np.searchsorted(sl.t, t_hi, side="right"))
        out.append((i, j, t_hi))
        i, t = j, t_hi
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_window(sl, i, j, t_hi, W, H, TXY):
    """The packet's encodings against the window's events, from scratch."""
    T, X, Y = TXY
    lo = int(np.searchsorted(sl.t, t_hi - WIN, side="left"))
    K = np.arange(i - lo, j - lo, dtype=np.int64)
    return oracle.encode_pooled(sl.x[lo:j], sl.y[lo:j], sl.t[lo:j], int(sl.t[lo]), W, H, D, 10, 10,
                                16_000.0, T, X, Y, K=K)[0]


def test_stream_packets_match_oracle_and_sums_do_not_drift():
    W, H = 128, 96
    sl = _long_stream(W, H, 30_000, 200_000, 3)
    rng = np.random.default_rng(1)
    enc, TXY, w = _enc(W, H)
    st = vk.Stream(enc, WIN, 40_000)
    pk = _packets(sl, rng)
    assert len(pk) > 40
    for q, (i, j, t_hi) in enumerate(pk):
        if j == i:
            st.push(_dev(sl.x[:0]), _dev(sl.y[:0]), _dev(sl.t[:0].view(np.int32)), t_hi,
                    predict=False)
            continue
        emb = st.push(_dev(sl.x[i:j]), _dev(sl.y[i:j]), _dev(sl.t[i:j].view(np.int32)), t_hi,
                      predict=False).cpu().numpy()
        if q % 7 == 0 or q == len(pk) - 1:
            ref = _oracle_window(sl, i, j, t_hi, W, H, TXY)
            assert emb_rel_err(emb, ref).max() <= EMB_TOL_FP32, q
    enc.sync_status()
    acc, cnt = st.accumulator()
    # a fresh stream given only the final window's events, as one packet
    t_hi = pk[-1][2]
    lo = int(np.searchsorted(sl.t, t_hi - WIN, side="left"))
    fresh = vk.Stream(enc, WIN, 40_000)
    fresh.push(_dev(sl.x[lo:]), _dev(sl.y[lo:]), _dev(sl.t[lo:].view(np.int32)), t_hi,
               predict=False)
    acc2, cnt2 = fresh.accumulator()
    assert st.window_events() == fresh.window_events() == len(sl.t) - lo
    assert np.array_equal(cnt, cnt2)
    assert np.array_equal(acc, acc2)  # exact fixed point: bit for bit
    st.close()
    fresh.close()


@pytest.mark.parametrize("mode", [vk.MLP_FP32, vk.MLP_FP16 | vk.ACC_FP16])
def test_stream_flows_match_oracle(mode):
    W, H = 160, 120
    sl = _long_stream(W, H, 20_000, 100_000, 4)
    rng = np.random.default_rng(2)
    enc, TXY, w = _enc(W, H, mode)
    st = vk.Stream(enc, WIN, 30_000)
    for q, (i, j, t_hi) in enumerate(_packets(sl, rng, 5_000)):
        if j == i:
            continue
        f = st.push(_dev(sl.x[i:j]), _dev(sl.y[i:j]), _dev(sl.t[i:j].view(np.int32)), t_hi).cpu().numpy()
        if q % 5 == 2:
            ref = _oracle_window(sl, i, j, t_hi, W, H, TXY)
            fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
            assert within_half_bound(f, fref, ref, w, mode) <= 1.0
    enc.sync_status()
    st.close()


def test_stream_rejects_out_of_window_and_unsorted_events_and_overflow():
    W, H = 64, 48
    sl = _long_stream(W, H, 3_000, 60_000, 5)
    enc, TXY, w = _enc(W, H)
    st = vk.Stream(enc, WIN, 2_500)
    j = int(np.searchsorted(sl.t, sl.t[0] + 20_000))
    t_hi = int(sl.t[j - 1]) + 1
    t_lo = t_hi - WIN
    x, y, t = sl.x[:j].copy(), sl.y[:j].copy(), sl.t[:j].copy()
    x[3] = W          # off the sensor
    t[5] = t_lo - 1   # before the window (and earlier than its predecessor)
    f = st.push(_dev(x), _dev(y), _dev(t.view(np.int32)), t_hi).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert np.all(f[3] == 0) and np.all(f[5] == 0)
    keep = np.setdiff1d(np.arange(j), [3, 5])
    assert st.window_events() == keep.size
    T, X, Y = TXY
    ref = oracle.encode_pooled(x[keep], y[keep], t[keep], int(t[0]), W, H, D, 10, 10, 16_000.0,
                               T, X, Y)[0]
    fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
    assert flow_rel_err(f[keep], fref, FLOW_FLOOR).max() <= FLOW_TOL[vk.MLP_FP32]
    st.close()
    # a packet inside one window that overflows a 500-event ring: its last
    # events are dropped and reported
    small = vk.Stream(enc, WIN, 500)
    assert int(sl.t[799]) - int(sl.t[0]) < WIN
    small.push(_dev(sl.x[:400]), _dev(sl.y[:400]), _dev(sl.t[:400].view(np.int32)),
               int(sl.t[399]) + 1)
    enc.sync_status()
    f2 = small.push(_dev(sl.x[400:800]), _dev(sl.y[400:800]), _dev(sl.t[400:800].view(np.int32)),
                    int(sl.t[799]) + 1).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_EBUSY
    assert small.window_events() == 500
    assert np.all(f2[100:] == 0) and np.any(f2[0] != 0)
    small.close()


def test_empty_pushes_slide_the_window():
    W, H = 64, 48
    sl = _long_stream(W, H, 2_000, 30_000, 6)
    enc, TXY, w = _enc(W, H)
    st = vk.Stream(enc, WIN, 4_000)
    t_hi = int(sl.t[-1]) + 1
    st.push(_dev(sl.x), _dev(sl.y), _dev(sl.t.view(np.int32)), t_hi, predict=False)
    assert st.window_events() == sl.n
    z16 = torch.empty(0, dtype=torch.int16, device="cuda")
    z32 = torch.empty(0, dtype=torch.int32, device="cuda")
    st.push(z16, z16, z32, t_hi + 10_000, predict=False)
    left = int(np.sum(sl.t >= t_hi + 10_000 - WIN))
    assert st.window_events() == left
    st.push(z16, z16, z32, t_hi + WIN + 1, predict=False)
    assert st.window_events() == 0
    acc, cnt = st.accumulator()
    assert not acc.any() and not cnt.any()  # everything left: exactly zero
    enc.sync_status()
    st.close()


def test_stream_keeps_time_order_within_and_across_packets():
    # [10, 100, 50, 60]: 50 and 60 come after 100 and are both rejected; a
    # packet whose first events are earlier than the last accepted one loses
    # exactly those; a push whose t_hi goes back is refused on the host
    W, H = 64, 48
    enc, TXY, w = _enc(W, H)
    st = vk.Stream(enc, WIN, 1_000)
    base = 1_000_000
    x = np.array([5, 6, 7, 8], np.int16)
    y = np.array([9, 9, 9, 9], np.int16)
    t = np.array([base + 10, base + 100, base + 50, base + 60], np.uint32)
    e1 = st.push(_dev(x), _dev(y), _dev(t.view(np.int32)), base + 200, predict=False).cpu().numpy()
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ERANGE
    assert st.window_events() == 2
    assert np.all(e1[2] == 0) and np.all(e1[3] == 0)
    T, X, Y = TXY
    ref = oracle.encode_pooled(x[:2], y[:2], t[:2], base, W, H, D, 10, 10, 16_000.0, T, X, Y)[0]
    assert emb_rel_err(e1[:2], ref).max() <= EMB_TOL_FP32
    # the next packet starts before 100, the last accepted time
    x2 = np.array([10, 11, 12, 13], np.int16)
    y2 = np.array([20, 20, 20, 20], np.int16)
    t2 = np.array([base + 90, base + 99, base + 100, base + 150], np.uint32)
    e2 = st.push(_dev(x2), _dev(y2), _dev(t2.view(np.int32)), base + 300, predict=False).cpu().numpy()
    with pytest.raises(vk.VeckmError):
        enc.sync_status()
    assert st.window_events() == 4
    assert np.all(e2[0] == 0) and np.all(e2[1] == 0)
    xs = np.concatenate([x[:2], x2[2:]])
    ys = np.concatenate([y[:2], y2[2:]])
    ts = np.concatenate([t[:2], t2[2:]])
    ref = oracle.encode_pooled(xs, ys, ts, base, W, H, D, 10, 10, 16_000.0, T, X, Y,
                               K=np.array([2, 3], np.int64))[0]
    assert emb_rel_err(e2[2:], ref).max() <= EMB_TOL_FP32
    # the ring's sums equal those of its four events built afresh
    acc, cnt = st.accumulator()
    fresh = vk.Stream(enc, WIN, 1_000)
    fresh.push(_dev(xs), _dev(ys), _dev(ts.view(np.int32)), base + 300, predict=False)
    enc.sync_status()
    acc2, cnt2 = fresh.accumulator()
    assert np.array_equal(cnt, cnt2) and np.array_equal(acc, acc2)
    with pytest.raises(vk.VeckmError) as ei:
        st.push(_dev(x2[:0]), _dev(y2[:0]), _dev(t2[:0].view(np.int32)), base + 299, predict=False)
    assert ei.value.status == vk.VECKM_EINVAL
    st.close()
    fresh.close()
