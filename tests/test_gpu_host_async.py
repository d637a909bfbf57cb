"""GPU tests of the pipelined host-buffer predict: calls with two in flight
return the FP64 oracle's flows (Eq. 6) for each slice, in order, and each
ticket reports the errors of its own call only."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import FLOW_FLOOR, FLOW_TOL, flow_rel_err, make, within_half_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

W, H, D = 200, 150, 64


def _pinned(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else a.view(dtype))
    return torch.from_numpy(a).pin_memory()


def _host(sl):
    return _pinned(sl.x), _pinned(sl.y), _pinned(sl.t, np.int32)


def _ref(sl, TXY, w, K=None):
    """(flows, encodings) of the FP64 oracle."""
    T, X, Y = TXY
    e = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, W, H, D, 10, 10, 16_000.0, T, X, Y, K=K)[0]
    return oracle.mlp(e, w.W1, w.b1, w.W2, w.b2), e


def test_pipelined_calls_match_oracle_in_order():
    # slices of growing and shrinking sizes (the staging slots are regrown),
    # every other one with a subset K
    sizes = [3_000, 9_000, 1_200, 12_000, 500, 7_000, 7_000]
    sls = [synth.event_slice(W, H, n, 20_000, n_edges=6, seed=70 + i) for i, n in enumerate(sizes)]
    enc, TXY, w = make(sls[0], D, t_span_us=20_000)
    rng = np.random.default_rng(9)
    Ks = [None if i % 2 == 0 else np.sort(rng.integers(0, s.n, s.n // 3)).astype(np.int64)
          for i, s in enumerate(sls)]
    outs = []
    tickets = []
    for i, sl in enumerate(sls):
        x, y, t = _host(sl)
        K = None if Ks[i] is None else _pinned(Ks[i])
        tk, out = enc.predict_host_async(x, y, t, sl.t_ref, K=K)
        tickets.append(tk)
        outs.append(out)
        if i >= 1:
            enc.host_wait(tickets[i - 1])
    enc.host_wait(tickets[-1])
    assert tickets == list(range(tickets[0], tickets[0] + len(sls)))
    for sl, K, out in zip(sls, Ks, outs):
        fref, eref = _ref(sl, TXY, w, K)
        assert out.shape == fref.shape
        assert flow_rel_err(out.numpy(), fref, FLOW_FLOOR).max() <= FLOW_TOL[vk.MLP_FP32]
    # the synchronous host call agrees with the pipelined one
    x, y, t = _host(sls[2])
    sync = enc.predict_host(x, y, t, sls[2].t_ref).numpy()
    assert np.abs(sync - outs[2].numpy()).max() <= 1e-5 * np.abs(sync).max()
    enc.sync_status()
    enc.close()


def test_each_ticket_reports_its_own_errors():
    sl = synth.event_slice(W, H, 2_000, 20_000, seed=80)
    enc, TXY, w = make(sl, D, t_span_us=20_000)
    bad = sl.x.copy()
    bad[7] = W  # off the sensor
    x, y, t = _host(sl)
    xb = _pinned(bad)
    t0, o0 = enc.predict_host_async(x, y, t, sl.t_ref)
    t1, o1 = enc.predict_host_async(xb, y, t, sl.t_ref)
    t2, o2 = enc.predict_host_async(x, y, t, sl.t_ref)
    enc.host_wait(t0)
    with pytest.raises(vk.VeckmError) as ei:
        enc.host_wait(t1)
    assert ei.value.status == vk.VECKM_ERANGE
    enc.host_wait(t2)
    # a ticket's status is kept: waiting again reports the same
    with pytest.raises(vk.VeckmError):
        enc.host_wait(t1)
    enc.host_wait(t0)
    fref, eref = _ref(sl, TXY, w)
    for o in (o0, o2):
        assert flow_rel_err(o.numpy(), fref, FLOW_FLOOR).max() <= FLOW_TOL[vk.MLP_FP32]
    f1 = o1.numpy()
    assert np.all(f1[7] == 0) and np.any(f1[8] != 0)
    # the context's own error word was left clear
    enc.sync_status()
    # unknown tickets, and tickets too old to report
    with pytest.raises(vk.VeckmError) as ei:
        enc.host_wait(t2 + 1)
    assert ei.value.status == vk.VECKM_EINVAL
    last = t2
    for _ in range(70):
        last, _o = enc.predict_host_async(x, y, t, sl.t_ref)
    enc.host_wait(last)
    with pytest.raises(vk.VeckmError) as ei:
        enc.host_wait(t0)
    assert ei.value.status == vk.VECKM_EINVAL
    # argument errors come back at once, with no ticket issued
    with pytest.raises(vk.VeckmError) as ei:
        enc.predict_host_async(x, y, t, sl.t_ref, K=_pinned(np.zeros(3, np.int64)),
                               out=torch.empty((0, 2)))
    assert ei.value.status == vk.VECKM_EINVAL
    enc.close()


def test_empty_call_and_mlp_precision():
    sl = synth.event_slice(W, H, 4_000, 20_000, n_edges=6, seed=81)
    enc, TXY, w = make(sl, D, mode=vk.MLP_FP16, t_span_us=20_000)
    z16 = _pinned(np.zeros(0, np.int16))
    z32 = _pinned(np.zeros(0, np.int32))
    tk, out = enc.predict_host_async(z16, z16, z32, 0)
    enc.host_wait(tk)
    assert out.shape == (0, 2)
    x, y, t = _host(sl)
    tk, out = enc.predict_host_async(x, y, t, sl.t_ref)
    enc.host_wait(tk)
    fref, eref = _ref(sl, TXY, w)
    assert within_half_bound(out.numpy(), fref, eref, w, vk.MLP_FP16) <= 1.0
    enc.close()
