"""veckm_encode_noalloc through the C ABI, against the FP64 oracle and against
veckm_encode.

veckm_encode_noalloc serves callers that may not allocate device memory
while a call runs: a loop with a real-time budget, which cannot wait for an
allocation and the synchronisation before it, or a process that reserves
all of a device's memory up front for its own allocator, where cudaMalloc
fails.  It keeps its per-event scratch in a fixed array that the library
declares statically.  Its result must match the oracle's pooled encoding
(Eq. 16-17) and veckm_encode's within the FP32 encoder bar, on consecutive
calls that reuse the shared array.  This file is collected last so that a
failure here never hides the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import EMB_TOL_FP32, emb_rel_err, make, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _noalloc(enc, x, y, t, t_ref, K, nK, out):
    st = vk.lib().veckm_encode_noalloc(enc.handle, _ptr(x), _ptr(y), _ptr(t), x.numel(),
                                       C.c_uint32(t_ref), _ptr(K), nK, _ptr(out),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_encode_matches_encode_on_consecutive_calls():
    import oracle
    sl = synth.event_slice(346, 260, 20_000, 10_000, n_edges=8, seed=314)
    enc, (T, X, Y), _ = make(sl, 64)
    x, y, t = to_dev(sl)
    ref = enc.encode(x, y, t, sl.t_ref).cpu().numpy().astype(np.float64)
    want = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, 64, 10, 10,
                                16_000.0, T, X, Y)[0]
    assert emb_rel_err(ref, want).max() <= EMB_TOL_FP32
    for _ in range(2):
        out = torch.full((sl.n, 128), float("nan"), dtype=torch.float32, device="cuda")
        assert _noalloc(enc, x, y, t, sl.t_ref, None, sl.n, out) == vk.VECKM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = emb_rel_err(got, ref)
        assert err.max() <= EMB_TOL_FP32, err.max()
        err = emb_rel_err(got, want)
        assert err.max() <= EMB_TOL_FP32, err.max()
    # an explicit subset K, after a call of another size
    K = torch.arange(3, sl.n, 11, dtype=torch.int64, device="cuda")
    out = torch.empty((K.numel(), 128), dtype=torch.float32, device="cuda")
    assert _noalloc(enc, x, y, t, sl.t_ref, K, K.numel(), out) == vk.VECKM_OK
    torch.cuda.synchronize()
    Kh = K.cpu().numpy()
    assert emb_rel_err(out.cpu().numpy(), ref[Kh]).max() <= EMB_TOL_FP32
    assert emb_rel_err(out.cpu().numpy(), want[Kh]).max() <= EMB_TOL_FP32
    enc.sync_status()


def test_predict_after_noalloc_encode():
    # a tensor-core predict zeroes one grid for the next call; the no-alloc
    # encode in between writes both grids, and the predict after it must
    # not take either for zero
    import oracle
    from tests.common import within_half_bound
    sl = synth.event_slice(160, 120, 30_000, 20_000, n_edges=6, seed=315)
    sparse = synth.event_slice(160, 120, 12_000, 20_000, n_edges=3, seed=316)
    enc, (T, X, Y), w = make(sl, 64, mode=vk.MLP_FP16, t_span_us=20_000)
    x, y, t = to_dev(sl)
    enc.predict(x, y, t, sl.t_ref)
    out = torch.empty((sl.n, 128), dtype=torch.float32, device="cuda")
    assert _noalloc(enc, x, y, t, sl.t_ref, None, sl.n, out) == vk.VECKM_OK
    xs, ys, ts = to_dev(sparse)
    f = enc.predict(xs, ys, ts, sparse.t_ref).cpu().numpy()
    e = oracle.encode_pooled(sparse.x, sparse.y, sparse.t, sparse.t_ref, 160, 120, 64, 10, 10,
                             16_000.0, T, X, Y)[0]
    assert within_half_bound(f, oracle.mlp(e, w.W1, w.b1, w.W2, w.b2), e, w, vk.MLP_FP16) <= 1.0
    enc.sync_status()


def test_noalloc_encode_rejects_more_events_than_its_array():
    sl = synth.event_slice(64, 48, 100, 1_000, seed=2)
    enc, _, _ = make(sl, 64)
    n = (1 << 20) + 1
    x = torch.zeros(n, dtype=torch.int16, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty((1, 128), dtype=torch.float32, device="cuda")
    K = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _noalloc(enc, x, x, t, 0, K, 1, out) == vk.VECKM_EINVAL
    assert b"1048576" in vk.lib().veckm_last_error()
