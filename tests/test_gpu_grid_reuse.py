"""GPU tests of grid reuse between calls: the tensor-core head zeroes the
row-pass grid for the next call's per-pixel sums, so successive dense calls
alternate between the context's two grids and skip the clear.  Every path
that writes a grid otherwise (the FP32 and embedding gathers, the direct
window form, streams, captured plans, the autotuner, calls too small to
spread the clearing) must leave the next call correct.  Each result is
checked against the FP64 oracle (Eq. 16 and Eq. 6); slices alternate between
dense and sparse so that a stale sum left in a grid would show."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import (EMB_TOL_FP32, FLOW_FLOOR, FLOW_TOL, emb_rel_err, flow_rel_err, make,
                          to_dev, within_half_bound)

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

W, H, D = 160, 120, 64


def _sl(seed, n):
    return synth.event_slice(W, H, n, 20_000, n_edges=3 + seed % 5, frac_noise=0.1, seed=seed)


def _emb_ref(sl, TXY, K=None):
    T, X, Y = TXY
    return oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, W, H, D, 10, 10, 16_000.0, T, X, Y,
                                K=K)[0]


def _check_predict(enc, sl, TXY, w, mode, K=None):
    x, y, t = to_dev(sl)
    Kd = None if K is None else torch.from_numpy(K).cuda()
    f = enc.predict(x, y, t, sl.t_ref, K=Kd).cpu().numpy()
    e = _emb_ref(sl, TXY, K)
    fref = oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)
    if mode == vk.MLP_FP32:
        err = flow_rel_err(f, fref, FLOW_FLOOR)
        assert err.max() <= FLOW_TOL[mode], err.max()
    else:
        r = within_half_bound(f, fref, e, w, mode)
        assert r <= 1.0, r


@pytest.mark.parametrize("mode", [vk.MLP_FP16, vk.MLP_FP16 | vk.ACC_FP16, vk.MLP_BF16])
def test_successive_predicts_alternate_grids(mode):
    sizes = [40_000, 12_000, 30_000, 12_000, 25_000]
    sls = [_sl(200 + i, n) for i, n in enumerate(sizes)]
    enc, TXY, w = make(sls[0], D, mode=mode, t_span_us=20_000)
    for sl in sls:
        _check_predict(enc, sl, TXY, w, mode)
    enc.sync_status()
    enc.close()


def test_every_path_between_predicts_leaves_the_next_one_correct():
    mode = vk.MLP_FP16
    enc, TXY, w = make(_sl(300, 10), D, mode=mode, t_span_us=20_000)
    dense, sparse = _sl(301, 40_000), _sl(302, 12_000)

    def predict_pair():
        _check_predict(enc, dense, TXY, w, mode)
        _check_predict(enc, sparse, TXY, w, mode)

    predict_pair()
    # the embedding gather (no clearing) on the cleared grid
    x, y, t = to_dev(dense)
    emb = enc.encode(x, y, t, dense.t_ref).cpu().numpy()
    assert emb_rel_err(emb, _emb_ref(dense, TXY)).max() <= EMB_TOL_FP32
    predict_pair()
    # the direct window form writes only occupied pixels of the first grid
    enc.set_path(vk.PATH_DIRECT)
    K = np.arange(0, sparse.n, 97, dtype=np.int64)
    x, y, t = to_dev(sparse)
    f = enc.predict(x, y, t, sparse.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    e = _emb_ref(sparse, TXY, K)
    err = flow_rel_err(f, oracle.mlp(e, w.W1, w.b1, w.W2, w.b2), FLOW_FLOOR)
    assert err.max() <= FLOW_TOL[vk.MLP_FP32], err.max()
    enc.set_path(vk.PATH_AUTO)
    predict_pair()
    # the FP32 head (no clearing)
    enc.set_mlp_mode(vk.MLP_FP32)
    _check_predict(enc, dense, TXY, w, vk.MLP_FP32)
    enc.set_mlp_mode(mode)
    predict_pair()
    # a call with too few requests to spread the clearing over, then full calls
    _check_predict(enc, dense, TXY, w, mode, K=np.arange(0, dense.n, 4001, dtype=np.int64))
    predict_pair()
    # a stream push converts its sums into the grids
    st = vk.Stream(enc, 20_000, 50_000)
    x, y, t = to_dev(sparse)
    st.push(x, y, t, int(sparse.t.max()) + 1, predict=False)
    st.close()
    predict_pair()
    # a captured plan holds two graphs with the grids' roles swapped and
    # replays the one whose sums go to the zeroed grid: back-to-back
    # replays, replays between predicts, and after paths that dirty both
    plan = enc.plan([vk.Slice(x, y, t, sparse.t_ref, W, H)])
    e = _emb_ref(sparse, TXY)
    fref = oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)
    for step in range(6):
        got = plan.launch().cpu().numpy()
        assert within_half_bound(got, fref, e, w, mode) <= 1.0, step
        if step == 2:
            predict_pair()
        if step == 4:
            x2, y2, t2 = to_dev(dense)
            enc.encode(x2, y2, t2, dense.t_ref)
    plan.close()
    predict_pair()
    enc.autotune(W, H)
    predict_pair()
    # pipelined host calls run on the context's own streams
    tk, out = enc.predict_host_async(torch.from_numpy(dense.x).pin_memory(),
                                     torch.from_numpy(dense.y).pin_memory(),
                                     torch.from_numpy(dense.t.view(np.int32)).pin_memory(),
                                     dense.t_ref)
    enc.host_wait(tk)
    e = _emb_ref(dense, TXY)
    assert within_half_bound(out.numpy(), oracle.mlp(e, w.W1, w.b1, w.W2, w.b2), e, w, mode) <= 1.0
    predict_pair()
    enc.sync_status()
    enc.close()


def test_rows_left_by_earlier_slices_are_never_read():
    # The pixel-sum grid is not cleared between calls after the bucket sort:
    # rows of pixels without events keep whatever an earlier slice left.
    # Slices with disjoint occupancy follow one another on one context, one
    # of them with a bucket above its shared-memory stage (records placed
    # straight into the bucket's region) and one that puts a pixel across
    # many record ranges; each result is checked against the oracle.
    mode = vk.MLP_FP16
    dense = _sl(401, 40_000)
    rng = np.random.default_rng(9)
    m = 12_000  # the first 32 pixels of row 0: about 12,000 records in one bucket
    hot = synth.EventSlice(rng.integers(0, 32, m).astype(np.int16), np.zeros(m, np.int16),
                           np.sort(rng.integers(dense.t_ref, dense.t_ref + 20_000, m)).astype(np.uint32),
                           np.ones(m, np.int8), W, H, dense.t_ref)
    one = 3_000  # a single pixel across about 24 ranges of 128 records
    single = synth.EventSlice(np.full(one, 77, np.int16), np.full(one, 50, np.int16),
                              np.sort(rng.integers(dense.t_ref, dense.t_ref + 20_000, one)).astype(np.uint32),
                              np.ones(one, np.int8), W, H, dense.t_ref)
    enc, TXY, w = make(dense, D, mode=mode, t_span_us=20_000)
    for sl in (dense, hot, dense, single, hot, _sl(402, 15_000)):
        _check_predict(enc, sl, TXY, w, mode)
        x, y, t = to_dev(sl)
        emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
        assert emb_rel_err(emb, _emb_ref(sl, TXY)).max() <= EMB_TOL_FP32
    enc.sync_status()
    enc.close()
