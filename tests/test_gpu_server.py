"""GPU tests of the serving loop: admission by device memory, packets served
alone and in a mix of streams give the same flows, ring wrap-around, error
attribution and the latency statistics."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import FLOW_FLOOR, flow_rel_err, within_half_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

D = 64
SPAN = 16_000
RES = [(346, 260), (640, 480), (128, 96), (97, 61)]


def _server(W=2048, H=1024, mode=vk.MLP_FP32, **kw):
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=W, height=H, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=SPAN)
    return vk.Server(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode, **kw), (T, X, Y), w


def _packet(i, n, res=None):
    W, H = res or RES[i % len(RES)]
    return synth.event_slice(W, H, n, SPAN, n_edges=3, frac_noise=0.1, seed=500 + i,
                             t0_us=10_000_000 + 16_000 * i)


def _pinned(sl):
    x = torch.from_numpy(sl.x).pin_memory()
    y = torch.from_numpy(sl.y).pin_memory()
    t = torch.from_numpy(sl.t.view(np.int32)).pin_memory()
    out = torch.zeros((sl.n, 2), dtype=torch.float32).pin_memory()
    return x, y, t, out


def _submit(srv, stream_id, sl, tag):
    x, y, t, out = _pinned(sl)
    assert srv.submit(stream_id, x, y, t, sl.t_ref, sl.width, sl.height, out, tag=tag)
    return out


def _all(srv, k):
    got = []
    while len(got) < k:
        got += srv.poll(wait_ms=2000)
    return {c["tag"]: c for c in got}


def test_a_packet_alone_and_in_a_mix_of_streams_gives_the_same_flows():
    # a 200 ms batching window: packets submitted together share one batch
    srv, TXY, w = _server(batch_window_us=200_000)
    P = _packet(0, 6_000, (346, 260))
    alone = _submit(srv, 3, P, tag=1)
    srv.drain()
    c = _all(srv, 1)
    assert c[1]["status"] == vk.VECKM_OK and c[1]["batch_packets"] == 1
    others = [_packet(i, 1_000 + 700 * i) for i in range(1, 9)]
    bufs = [_pinned(sl) for sl in others]
    pb = _pinned(P)
    outs = {}
    for i, (sl, b) in enumerate(zip(others, bufs)):
        if i == 4:
            assert srv.submit(3, *pb[:3], P.t_ref, P.width, P.height, pb[3], tag=2)
        assert srv.submit(10 + i, *b[:3], sl.t_ref, sl.width, sl.height, b[3], tag=10 + i)
        outs[10 + i] = b[3]
    mixed = pb[3]
    srv.drain()
    c = _all(srv, 9)
    assert all(v["status"] == vk.VECKM_OK for v in c.values())
    assert c[2]["batch_packets"] == 9  # P shared its batch with eight other streams
    a, m = alone.numpy(), mixed.numpy()
    assert np.abs(a - m).max() <= 1e-5 * np.abs(a).max()
    T, X, Y = TXY
    ref = oracle.encode_pooled(P.x, P.y, P.t, P.t_ref, P.width, P.height, D, 10, 10, 16_000.0,
                               T, X, Y)[0]
    fref = oracle.mlp(ref, w.W1, w.b1, w.W2, w.b2)
    assert flow_rel_err(m, fref, FLOW_FLOOR).max() <= 1e-4
    for i, sl in enumerate(others):
        r = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                 16_000.0, T, X, Y)[0]
        f = oracle.mlp(r, w.W1, w.b1, w.W2, w.b2)
        assert flow_rel_err(outs[10 + i].numpy(), f, FLOW_FLOOR).max() <= 1e-4
    st = srv.stats()
    assert st["completed"] == st["admitted"] == 10 and st["refused"] == 0
    assert st["streams"] == 9 and st["events_completed"] == 2 * P.n + sum(s.n for s in others)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_admission_by_device_memory():
    # an arena of 64 KiB: 8 bytes per event (three 256-byte aligned arrays)
    srv, _, _ = _server(arena_bytes=64 * 1024)
    big = _packet(1, 10_000)
    x, y, t, out = _pinned(big)
    assert not srv.submit(0, x, y, t, big.t_ref, big.width, big.height, out)  # never fits
    small = [_packet(i, 1_500) for i in range(12)]
    admitted = 0
    bufs = []
    for i, sl in enumerate(small):
        x, y, t, out = _pinned(sl)
        bufs.append(out)
        admitted += srv.submit(i, x, y, t, sl.t_ref, sl.width, sl.height, out, tag=100 + i)
    srv.drain()
    st = srv.stats()
    assert st["submitted"] == 13 and st["admitted"] == admitted and st["refused"] == 13 - admitted
    assert 1 <= admitted <= 12 and st["completed"] == admitted
    # with the arena empty again a packet that fits is admitted
    x, y, t, out = _pinned(small[0])
    assert srv.submit(0, x, y, t, small[0].t_ref, small[0].width, small[0].height, out)
    srv.drain()
    srv.close()


def test_ring_wraps_around_and_every_packet_stays_correct():
    # packets of uneven sizes through a 160 KiB arena, one at a time so the ring
    # wraps many times; each packet's flows equal the single-slice call's
    srv, TXY, w = _server(arena_bytes=160 * 1024)
    T, X, Y = TXY
    ref_enc = {}
    rng = np.random.default_rng(3)
    for i in range(14):
        sl = _packet(20 + i, int(rng.integers(500, 5_000)))
        out = _submit(srv, i % 5, sl, tag=i)
        c = _all(srv, 1)
        assert c[i]["status"] == vk.VECKM_OK
        key = (sl.width, sl.height)
        if key not in ref_enc:
            p = vk.Params(width=sl.width, height=sl.height, D=D, dx=10, dy=10, dt_us=16_000,
                          t_span_us=SPAN)
            ref_enc[key] = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y)
        xd = torch.from_numpy(sl.x).cuda()
        yd = torch.from_numpy(sl.y).cuda()
        td = torch.from_numpy(sl.t.view(np.int32)).cuda()
        f1 = ref_enc[key].predict(xd, yd, td, sl.t_ref).cpu().numpy()
        assert np.abs(out.numpy() - f1).max() <= 1e-5 * np.abs(f1).max(), i
    srv.close()


def test_an_out_of_range_event_is_reported_on_its_packet():
    srv, _, _ = _server()
    good = _packet(40, 2_000)
    bad = _packet(41, 2_000, (128, 96))
    bad.x[11] = 128  # outside its own sensor
    out_g = _submit(srv, 1, good, tag=1)
    srv.drain()
    out_b = _submit(srv, 2, bad, tag=2)
    srv.drain()
    c = _all(srv, 2)
    assert c[1]["status"] == vk.VECKM_OK and c[2]["status"] == vk.VECKM_ERANGE
    assert np.all(out_b.numpy()[11] == 0)
    srv.close()


def test_malformed_packets_are_rejected():
    srv, _, _ = _server(W=512, H=512)
    sl = _packet(50, 100, (600, 100))
    x, y, t, out = _pinned(sl)
    with pytest.raises(vk.VeckmError) as ei:
        srv.submit(0, x, y, t, sl.t_ref, 600, 100, out)  # wider than the canvas
    assert ei.value.status == vk.VECKM_EINVAL
    with pytest.raises(vk.VeckmError):
        srv.submit(70_000, x, y, t, sl.t_ref, 100, 100, out)  # stream id out of range
    srv.close()


# ------------------------------------------------------------ resident windows
WIN = 32_000  # 2 delta_t
SENS = [(128, 96), (97, 61), (160, 120)]


def _sensor_stream(i, n):
    W, H = SENS[i]
    return synth.event_slice(W, H, n, 150_000, n_edges=4, frac_noise=0.1, seed=700 + i,
                             t0_us=20_000_000)


def _cut(sl, rng, mean_us=4_000):
    """Consecutive packets of a sensor stream at random time boundaries
    (index ranges; every packet non-empty)."""
    out, i = [], 0
    t = int(sl.t[0])
    while i < sl.n:
        t += int(rng.integers(mean_us // 3, 2 * mean_us))
        j = int(np.searchsorted(sl.t, t, side="right"))
        if j > i:
            out.append((i, j))
            i = j
    return out


def _window_ref(sl, i, j, TXY, w):
    """The packet's flows against the window [t_hi - WIN, t_hi] of its stream
    (t_hi = its last event), recomputed from scratch by the oracle."""
    T, X, Y = TXY
    t_hi = int(sl.t[j - 1])
    lo = int(np.searchsorted(sl.t, t_hi - WIN, side="left"))
    K = np.arange(i - lo, j - lo, dtype=np.int64)
    e = oracle.encode_pooled(sl.x[lo:j], sl.y[lo:j], sl.t[lo:j], int(sl.t[lo]), sl.width,
                             sl.height, D, 10, 10, 16_000.0, T, X, Y, K=K)[0]
    return e, oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)


def _submit_range(srv, sid, sl, i, j, tag):
    x = torch.from_numpy(np.ascontiguousarray(sl.x[i:j])).pin_memory()
    y = torch.from_numpy(np.ascontiguousarray(sl.y[i:j])).pin_memory()
    t = torch.from_numpy(np.ascontiguousarray(sl.t[i:j]).view(np.int32)).pin_memory()
    out = torch.zeros((j - i, 2), dtype=torch.float32).pin_memory()
    assert srv.submit(sid, x, y, t, int(sl.t[i]), sl.width, sl.height, out, tag=tag)
    return out


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_FP32])
def test_resident_windows_alone_equal_mix_and_match_the_oracle(mode):
    """Each stream's packets slide its resident window; a stream's flows are
    bit-identical whether its packets run alone or interleaved with other
    streams' packets (on the device at the same time), and match the oracle
    recomputed on each packet's window."""
    streams = [_sensor_stream(i, 12_000 + 4_000 * i) for i in range(3)]
    rng = np.random.default_rng(17)
    cuts = [_cut(sl, rng) for sl in streams]
    kw = dict(W=512, H=512, mode=mode, window_us=WIN, window_capacity=60_000)
    # stream 0 alone
    srv, TXY, w = _server(**kw)
    alone = [_submit_range(srv, 5, streams[0], i, j, tag=q) for q, (i, j) in enumerate(cuts[0])]
    srv.drain()
    c = _all(srv, len(alone))
    assert all(v["status"] == vk.VECKM_OK for v in c.values())
    srv.close()
    # all three interleaved at random, each stream's packets in order
    srv, _, _ = _server(**kw)
    order = [s for s in range(3) for _ in cuts[s]]
    rng.shuffle(order)
    nxt = [0, 0, 0]
    outs = {}
    for s in order:
        q = nxt[s]
        nxt[s] += 1
        i, j = cuts[s][q]
        outs[(s, q)] = _submit_range(srv, 5 + s, streams[s], i, j, tag=1000 * s + q)
    srv.drain()
    c = _all(srv, len(order))
    assert all(v["status"] == vk.VECKM_OK for v in c.values())
    st = srv.stats()
    assert st["completed"] == st["admitted"] == len(order) and st["streams"] == 3
    for q in range(len(cuts[0])):
        assert np.array_equal(outs[(0, q)].numpy(), alone[q].numpy()), q
    for s in range(3):
        for q in range(0, len(cuts[s]), 5):
            i, j = cuts[s][q]
            e, fref = _window_ref(streams[s], i, j, TXY, w)
            f = outs[(s, q)].numpy()
            if mode == vk.MLP_FP32:
                assert flow_rel_err(f, fref, FLOW_FLOOR).max() <= 1e-4, (s, q)
            else:
                assert within_half_bound(f, fref, e, w, mode) <= 1.0, (s, q)
    srv.close()


def test_resident_windows_refuse_a_stream_whose_state_cannot_be_allocated():
    sl = _sensor_stream(0, 6_000)
    srv, TXY, w = _server(W=512, H=512, mode=vk.MLP_FP16, window_us=WIN, window_capacity=20_000)
    cuts = _cut(sl, np.random.default_rng(4))
    i, j = cuts[0]
    x = torch.from_numpy(np.ascontiguousarray(sl.x[i:j])).pin_memory()
    y = torch.from_numpy(np.ascontiguousarray(sl.y[i:j])).pin_memory()
    t = torch.from_numpy(np.ascontiguousarray(sl.t[i:j]).view(np.int32)).pin_memory()
    out = torch.zeros((j - i, 2), dtype=torch.float32).pin_memory()
    vk.debug_fail_alloc(3)  # the new stream's context fails to allocate
    try:
        assert not srv.submit(1, x, y, t, int(sl.t[i]), sl.width, sl.height, out)
    finally:
        vk.debug_fail_alloc(-1)
    # the next packet of the stream creates its state and is served
    assert srv.submit(1, x, y, t, int(sl.t[i]), sl.width, sl.height, out)
    srv.drain()
    c = _all(srv, 1)
    assert list(c.values())[0]["status"] == vk.VECKM_OK
    e, fref = _window_ref(sl, i, j, TXY, w)
    assert within_half_bound(out.numpy(), fref, e, w, vk.MLP_FP16) <= 1.0
    st = srv.stats()
    assert st["refused"] == 1 and st["admitted"] == 1
    # a stream may not change its sensor
    with pytest.raises(vk.VeckmError) as ei:
        srv.submit(1, x, y, t, int(sl.t[i]), 64, 48, out)
    assert ei.value.status == vk.VECKM_EINVAL
    srv.close()
