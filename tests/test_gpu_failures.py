"""GPU tests of failure detection, in the forms that fault and hang nothing.

- Bounded device waits: with a short wait limit and the stall injection, the
  tensor-core head's producers never signal a filled tile, so every wait of
  the head runs out; the call reports VECKM_ETIMEOUT and the same context
  then predicts correctly again (Eq. 6 against the FP64 oracle).
- Allocation failures (host-side injection): each device or pinned-host
  allocation of context creation, record growth, plan creation, stream
  creation and server creation is failed in turn; the call reports
  VECKM_ENOMEM, frees what it had allocated (free device memory returns to
  where it was) and leaves the context usable.
"""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import make, to_dev, within_half_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

D = 64
# device memory comes back to the driver in pages: allow a few of them
LEAK_SLACK = 8 << 20


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _oracle_flow(sl, TXY, w):
    T, X, Y = TXY
    e = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                             16_000.0, T, X, Y)[0]
    return e, oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_BF16 | vk.ACC_FP16])
def test_head_wait_runs_out_and_the_context_stays_usable(mode):
    sl = synth.event_slice(160, 120, 20_000, 20_000, n_edges=5, seed=901)
    enc, TXY, w = make(sl, D, mode=mode, t_span_us=20_000)
    x, y, t = to_dev(sl)
    enc.set_wait_limit(20_000_000)  # about 10 ms at 2 GHz
    enc.set_injection(vk.INJECT_HEAD_STALL)
    enc.predict(x, y, t, sl.t_ref)
    with pytest.raises(vk.VeckmError) as ei:
        enc.sync_status()
    assert ei.value.status == vk.VECKM_ETIMEOUT
    enc.sync_status()  # the error word was read and cleared
    enc.set_injection(vk.INJECT_NONE)
    enc.set_wait_limit(0)
    e, fref = _oracle_flow(sl, TXY, w)
    for _ in range(2):
        f = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
        enc.sync_status()
        assert within_half_bound(f, fref, e, w, mode) <= 1.0
    enc.close()


def test_injection_and_wait_limit_arguments():
    sl = synth.event_slice(64, 48, 500, 10_000, seed=902)
    enc, _, _ = make(sl, D, mode=vk.MLP_FP16)
    with pytest.raises(vk.VeckmError) as ei:
        enc.set_injection(7)
    assert ei.value.status == vk.VECKM_EINVAL
    with pytest.raises(vk.VeckmError) as ei:
        enc.set_wait_limit(-1)
    assert ei.value.status == vk.VECKM_EINVAL
    enc.close()


def _count_allocs(fn):
    vk.debug_fail_alloc(-1)
    out = fn()
    return vk.debug_fail_alloc(-1), out


def _fails_cleanly(fn, n_allocs):
    """Fails each of the n_allocs allocations of fn in turn: VECKM_ENOMEM, and
    the free device memory comes back to what it was."""
    assert n_allocs > 0
    for k in range(n_allocs):
        before = _free()
        vk.debug_fail_alloc(k)
        try:
            with pytest.raises(vk.VeckmError) as ei:
                fn()
        finally:
            vk.debug_fail_alloc(-1)
        assert ei.value.status == vk.VECKM_ENOMEM, (k, ei.value)
        assert before - _free() <= LEAK_SLACK, k


def test_context_creation_fails_each_allocation_cleanly():
    sl = synth.event_slice(200, 150, 3_000, 10_000, seed=903)
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=200, height=150, D=D, dt_us=16_000, t_span_us=10_000)

    def create():
        return vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=vk.MLP_FP16)

    n, enc = _count_allocs(create)
    enc.close()
    _fails_cleanly(lambda: create().close(), n)
    # after all that, a context works
    enc = create()
    x, y, t = to_dev(sl)
    f = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    enc.sync_status()
    e, fref = _oracle_flow(sl, (T, X, Y), w)
    assert within_half_bound(f, fref, e, w, vk.MLP_FP16) <= 1.0
    enc.close()


def test_record_growth_plan_and_stream_fail_cleanly_and_the_context_stays_usable():
    small = synth.event_slice(160, 120, 2_000, 20_000, seed=904)
    big = synth.event_slice(160, 120, 30_000, 20_000, n_edges=6, seed=905)
    enc, TXY, w = make(small, D, mode=vk.MLP_FP16, t_span_us=20_000)
    xs, ys, ts = to_dev(small)
    xb, yb, tb = to_dev(big)
    enc.predict(xs, ys, ts, small.t_ref)
    enc.sync_status()
    # the record buffers grow for the larger slice
    n, _ = _count_allocs(lambda: enc.predict(xb, yb, tb, big.t_ref))
    enc.sync_status()
    enc2, _, _ = make(small, D, mode=vk.MLP_FP16, t_span_us=20_000)
    enc2.predict(xs, ys, ts, small.t_ref)
    enc2.sync_status()
    _fails_cleanly(lambda: enc2.predict(xb, yb, tb, big.t_ref), n)
    f = enc2.predict(xb, yb, tb, big.t_ref).cpu().numpy()
    enc2.sync_status()
    e, fref = _oracle_flow(big, TXY, w)
    assert within_half_bound(f, fref, e, w, vk.MLP_FP16) <= 1.0
    enc2.close()
    # a captured plan (the first one also grows the context's batch buffers;
    # count the allocations of a second one)
    sl = [vk.Slice(xb, yb, tb, big.t_ref, 160, 120)]
    enc.plan(sl).close()
    n, plan = _count_allocs(lambda: enc.plan(sl))
    plan.close()
    _fails_cleanly(lambda: enc.plan(sl).close(), n)
    plan = enc.plan(sl)
    f = plan.launch().cpu().numpy()
    assert within_half_bound(f, fref, e, w, vk.MLP_FP16) <= 1.0
    plan.close()
    # a sliding-window stream
    n, st = _count_allocs(lambda: vk.Stream(enc, 32_000, 40_000))
    st.close()
    _fails_cleanly(lambda: vk.Stream(enc, 32_000, 40_000).close(), n)
    st = vk.Stream(enc, 32_000, 40_000)
    f = st.push(xb, yb, tb, int(big.t.max()) + 1).cpu().numpy()
    enc.sync_status()
    assert within_half_bound(f, fref, e, w, vk.MLP_FP16) <= 1.0
    st.close()
    enc.close()


def test_server_creation_fails_each_allocation_cleanly():
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=512, height=512, D=D, dt_us=16_000, t_span_us=16_000)

    def create():
        return vk.Server(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=vk.MLP_FP16,
                         arena_bytes=64 << 20, max_batch_events=1 << 20)

    n, srv = _count_allocs(create)
    srv.close()
    _fails_cleanly(lambda: create().close(), n)
    srv = create()
    sl = synth.event_slice(346, 260, 5_000, 16_000, n_edges=3, seed=906)
    hx = torch.from_numpy(sl.x).pin_memory()
    hy = torch.from_numpy(sl.y).pin_memory()
    ht = torch.from_numpy(sl.t.view(np.int32)).pin_memory()
    out = torch.zeros((sl.n, 2), dtype=torch.float32).pin_memory()
    assert srv.submit(0, hx, hy, ht, sl.t_ref, 346, 260, out)
    srv.drain()
    (c,) = srv.poll(16)
    assert c["status"] == vk.VECKM_OK
    e, fref = _oracle_flow(sl, (T, X, Y), w)
    assert within_half_bound(out.numpy(), fref, e, w, vk.MLP_FP16) <= 1.0
    srv.close()
