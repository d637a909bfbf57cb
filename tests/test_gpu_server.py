"""GPU tests of the serving loop: admission by device memory, packets served
alone and in a mix of streams give the same flows, ring wrap-around, error
attribution and the latency statistics."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import FLOW_FLOOR, flow_rel_err

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
