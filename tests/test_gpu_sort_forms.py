"""GPU tests of the sort by pixel that feeds the per-pixel sums (the bucket
form): a bucket holding more records than its shared-memory stage (placed
straight into its region instead), a slice of more than 4096 x 4096
events (tiles of 8192 events), and a slice beyond the bucket form's limits
(histogram, scan and placement).  Encodings are checked against the FP64
oracle's pooled form (Algorithm 1, Eq. 16-17) on the same events."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk
from tests.common import EMB_TOL_FP32, emb_rel_err, make, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

D = 64


def _ref(sl, TXY, K=None):
    T, X, Y = TXY
    return oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                16_000.0, T, X, Y, K=K)[0]


def test_bucket_above_its_stage():
    # 160 x 120 = 19200 pixels: buckets of 32 pixels; 12,000 extra events on
    # the first 32 pixels of row 0 put about 12,000 records in one bucket
    sl = synth.event_slice(160, 120, 6_000, 20_000, n_edges=5, seed=501)
    rng = np.random.default_rng(5)
    m = 12_000
    hot_x = rng.integers(0, 32, m).astype(np.int16)
    hot_t = np.sort(rng.integers(sl.t_ref, sl.t_ref + 20_000, m)).astype(np.uint32)
    x = np.concatenate([sl.x, hot_x])
    y = np.concatenate([sl.y, np.zeros(m, np.int16)])
    t = np.concatenate([sl.t, hot_t])
    big = synth.EventSlice(x, y, t, np.ones(x.size, np.int8), 160, 120, sl.t_ref)
    enc, TXY, _ = make(big, D, t_span_us=20_000)
    xd, yd, td = to_dev(big)
    emb = enc.encode(xd, yd, td, big.t_ref).cpu().numpy()
    assert emb_rel_err(emb, _ref(big, TXY)).max() <= EMB_TOL_FP32
    enc.sync_status()


def test_more_events_than_one_round_of_tiles():
    # 17 M events (more than 4096 tiles of 4096): tiles of 8192 events; a
    # sample of requested events against the oracle
    n = 17_000_000
    sl = synth.event_slice(160, 120, n, 20_000, n_edges=6, seed=502)
    enc, TXY, _ = make(sl, D, t_span_us=20_000)
    x, y, t = to_dev(sl)
    K = np.sort(np.random.default_rng(6).choice(n, 2_000, replace=False)).astype(np.int64)
    emb = enc.encode(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    assert emb_rel_err(emb, _ref(sl, TXY, K)).max() <= EMB_TOL_FP32
    enc.sync_status()


def test_histogram_sort_above_the_bucket_limits():
    # 34 M events (more than 2 x 4096 tiles of 8192): the histogram, scan and
    # placement form of the sort, whose exclusive prefix gives the row
    # offsets of the per-pixel sums; dense path forced for the sampled requests
    n = 34_000_000
    sl = synth.event_slice(160, 120, n, 20_000, n_edges=6, seed=503)
    enc, TXY, _ = make(sl, D, t_span_us=20_000)
    enc.set_path(vk.PATH_DENSE)
    x, y, t = to_dev(sl)
    K = np.sort(np.random.default_rng(7).choice(n, 1_000, replace=False)).astype(np.int64)
    emb = enc.encode(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    assert enc.last_path() == vk.PATH_DENSE
    assert emb_rel_err(emb, _ref(sl, TXY, K)).max() <= EMB_TOL_FP32
    enc.sync_status()
