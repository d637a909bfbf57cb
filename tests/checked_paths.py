"""Run in a fresh process with VECKM_LIBRARY=checked (tests/test_gpu_checked.py):
the main paths of the library on the bounds-checked build, each against the
FP64 oracle, then the number of indices that would have left their buffer
(veckm_debug_checks) printed as `CHECKS <count> <where>`."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2504_19417_gb300 import synth  # noqa: E402
from paper_2504_19417_gb300 import veckm as vk  # noqa: E402
from tests.common import (EMB_TOL_FP32, FLOW_TOL_FP32, emb_rel_err, flow_rel_err, make,  # noqa: E402
                          to_dev, within_half_bound)

assert os.environ.get("VECKM_LIBRARY") == "checked"
assert vk.debug_checks() == (0, 0)  # loads the checked library (the call fails in the normal one)


def refs(sl, D, TXY, w, K=None):
    T, X, Y = TXY
    e = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                             16_000.0, T, X, Y, K=K)[0]
    return e, oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)


# 1. one slice, D = 64: embeddings, the plain head and the three tensor-core
# modes (sorted records), and explicit requests
sl = synth.event_slice(200, 150, 30_000, 20_000, n_edges=6, seed=71)
D = 64
x, y, t = to_dev(sl)
for mode in (vk.MLP_FP32, vk.MLP_FP16, vk.MLP_BF16, vk.MLP_FP16 | vk.ACC_FP16):
    enc, TXY, w = make(sl, D, mode=mode, t_span_us=20_000)
    e_ref, f_ref = refs(sl, D, TXY, w)
    emb = enc.encode(x, y, t, sl.t_ref).cpu().numpy()
    assert emb_rel_err(emb, e_ref).max() <= EMB_TOL_FP32
    f = enc.predict(x, y, t, sl.t_ref).cpu().numpy()
    if mode == vk.MLP_FP32:
        assert flow_rel_err(f, f_ref).max() <= FLOW_TOL_FP32
    else:
        assert within_half_bound(f, f_ref, e_ref, w, mode) <= 1.0
    K = np.sort(np.random.default_rng(1).choice(sl.n, 3_000, replace=False)).astype(np.int64)
    fk = enc.predict(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
    assert np.allclose(fk, f[K], rtol=0, atol=1e-4 * (1 + np.abs(f[K]).max()))
    enc.sync_status()
    enc.close()

# 2. D = 128 (the shared-memory operand head) on a wider sensor
sl2 = synth.event_slice(320, 180, 40_000, 20_000, n_edges=6, seed=72)
enc, TXY, w = make(sl2, 128, mode=vk.MLP_FP16, t_span_us=20_000)
x2, y2, t2 = to_dev(sl2)
e_ref, f_ref = refs(sl2, 128, TXY, w)
f = enc.predict(x2, y2, t2, sl2.t_ref).cpu().numpy()
assert within_half_bound(f, f_ref, e_ref, w, vk.MLP_FP16) <= 1.0
enc.sync_status()
enc.close()

# 3. a sliding-window stream fed the first slice in two packets
enc, TXY, w = make(sl, D, mode=vk.MLP_FP16, t_span_us=20_000)
st = vk.Stream(enc, 32_000, 40_000)
half = sl.n // 2
st.push(x[:half], y[:half], t[:half], int(sl.t[half - 1]) + 1)
f = st.push(x[half:], y[half:], t[half:], int(sl.t.max()) + 1).cpu().numpy()
e_ref, f_ref = refs(sl, D, TXY, w)
assert within_half_bound(f, f_ref[half:], e_ref[half:], w, vk.MLP_FP16) <= 1.0
enc.sync_status()
st.close()

# 4. a batch of two slices on a context large enough for their canvas, and
# the direct window form
sl3 = synth.event_slice(120, 90, 8_000, 20_000, n_edges=4, seed=73)
x3, y3, t3 = to_dev(sl3)
T, X, Y = TXY
pb = vk.Params(width=512, height=256, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=20_000)
encb = vk.Encoder(pb, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=vk.MLP_FP16)
fb = encb.predict_batch([vk.Slice(x, y, t, sl.t_ref, sl.width, sl.height),
                         vk.Slice(x3, y3, t3, sl3.t_ref, sl3.width, sl3.height)]).cpu().numpy()
e3, f3 = refs(sl3, D, TXY, w)
assert within_half_bound(fb[: sl.n], f_ref, e_ref, w, vk.MLP_FP16) <= 1.0
assert within_half_bound(fb[sl.n:], f3, e3, w, vk.MLP_FP16) <= 1.0
encb.sync_status()
encb.close()
enc.set_mlp_mode(vk.MLP_FP32)
enc.set_path(vk.PATH_DIRECT)
K = np.sort(np.random.default_rng(2).choice(sl.n, 500, replace=False)).astype(np.int64)
fd = enc.predict(x, y, t, sl.t_ref, K=torch.from_numpy(K).cuda()).cpu().numpy()
_, fdr = refs(sl, D, TXY, w, K=K)
assert flow_rel_err(fd, fdr).max() <= FLOW_TOL_FP32
enc.sync_status()
enc.close()

n, where = vk.debug_checks()
print("CHECKS", n, where, flush=True)
