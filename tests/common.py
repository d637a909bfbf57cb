"""Helpers shared by the GPU tests: build a context from seeded inputs, move a
slice to the device, and the error measures the parity bars are stated in."""
import numpy as np

from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk

# Parity bars:
#  - FP32 encoder: per requested event, ||emb_gpu - emb_ref||_2 / ||emb_ref||_2.
#  - FP32 flows: per event ||flow_gpu - flow_ref||_2 / max(||flow_ref||_2, floor)
#    with floor = FLOW_FLOOR * median ||flow_ref||_2.  The FP32 error of a flow
#    is absolute, not relative: the encoding carries ~1e-6 relative error, and
#    the perceptron sums 2D + 1 and 129 signed terms whose magnitudes are about
#    ten times the flow's, so a flow that cancels keeps the error of its terms.
#    Measured on 60,000-event 640x480 slices of the four recipes (Section 2.3):
#    at most 7e-6 x median absolute; relative to max(|flow|, 1e-3 median) up to
#    6.9e-4, relative to max(|flow|, 0.05 median) at most 4.4e-5.  0.05 is the
#    tightest floor that holds the 1e-4 bar with room for the run-to-run
#    variation of FP32 summation order (about 25 %).
EMB_TOL_FP32 = 1e-4
FLOW_TOL_FP32 = 1e-4
FLOW_TOL = {vk.MLP_FP32: 1e-4}
FLOW_FLOOR = 0.05
FLOW_FLOOR_HALF = 0.25


def make(sl, D, dx=10, dy=10, dt_us=16_000, mode=vk.MLP_FP32, freq_seed=0, t_span_us=None):
    T, X, Y = synth.frequencies(D, freq_seed)
    w = synth.mlp_weights(D, 128, 3)
    span = t_span_us if t_span_us is not None else max(1, int(sl.t.max()) - sl.t_ref if sl.n else 1)
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=dx, dy=dy, dt_us=dt_us,
                  t_span_us=span)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    return enc, (T, X, Y), w


def to_dev(sl):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(sl.x)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(sl.y)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(sl.t).view(np.int32)).cuda()
    return x, y, t


def emb_rel_err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    num = np.linalg.norm(gpu - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return num / den


# unit roundoff of the first layer's operands; FP32 (the plain head) uses the
# same propagation bound with u = 2^-24, where the 1e-5 term (FP32
# accumulation and encoder error) dominates
UNIT_ROUNDOFF = {vk.MLP_FP32: 2.0 ** -24, vk.MLP_BF16: 2.0 ** -8, vk.MLP_FP16: 2.0 ** -11}


U16 = 2.0 ** -11  # FP16 unit roundoff (the second layer of the tensor-core head)


def _second_layer(emb_ref, w, dh):
    """Bound on what the tensor-core head's second layer adds: ReLU(h) and W2
    are each rounded once to FP16 (u16 = 2^-11; W2 entries below FP16's
    normal range lose at most 2^-25 absolute) and their products summed in
    FP32, and the first layer's error dh_j passes through W2 (ReLU is
    1-Lipschitz):
        sum_j |W2_oj| dh_j + sum_j ((2 u16 + u16^2) |W2_oj| + 2^-25) (ReLU(h_j) + dh_j)"""
    W1 = w.W1.astype(np.float64)
    W2 = np.abs(w.W2.astype(np.float64))
    relu_h = np.maximum(emb_ref @ W1.T + w.b1.astype(np.float64), 0.0)
    r = relu_h + dh
    return dh @ W2.T + r @ ((2 * U16 + U16 * U16) * W2 + 2.0 ** -25).T


def half_flow_bound(emb_ref, w, mode):
    """A-priori bound on |flow_gpu - flow_ref| per output for the tensor-core
    head.  First layer: operands (emb and W1) rounded to BF16/FP16 (unit
    roundoff u) and products accumulated in FP32, so each hidden unit is off
    by at most
        dh_j = (2u + u^2 + 1e-5) * sum_c |W1_jc e_c|
    (each rounded product is W e (1 + d1)(1 + d2); the 1e-5 covers FP32
    accumulation over at most 256 terms and the FP32 error of the encoder).
    Second layer: see _second_layer.  (MLP_FP32 uses the first-layer term
    alone with u = 2^-24.)"""
    u = UNIT_ROUNDOFF[mode & 3]
    dh = (2 * u + u * u + 1e-5) * (np.abs(emb_ref) @ np.abs(w.W1.astype(np.float64)).T)
    if mode == vk.MLP_FP32:
        return dh @ np.abs(w.W2.astype(np.float64)).T
    return _second_layer(emb_ref, w, dh)


def acc16_flow_bound(emb_ref, w, mode):
    """Bound for the FP16 pooled grid (VECKM_ACC_FP16) on top of the MMA operand
    rounding: the stored normalised pooled value p and the phase are each
    rounded once to FP16 (u_h = 2^-11) and the packed half2 product
    Re = p_r c + p_i s, Im = p_i c - p_r s adds a rounding per multiply and per
    fused add, so |d e_c| <= 4 u_h (|p_r| + |p_i|) <= 4 sqrt(2) u_h |p_d| < 6 u_h |e_d|
    for both columns c of channel d (|p_d| = |e_d|, the phase has modulus 1).
        dh_j = sum_c |W1_jc| (2 u |e_c| + 6 u_h |e_d(c)| + 1e-5 |e_c|)
    then the second layer as in _second_layer."""
    u = UNIT_ROUNDOFF[mode & 3]
    uh = 2.0 ** -11
    D = emb_ref.shape[1] // 2
    mag = np.hypot(emb_ref[:, :D], emb_ref[:, D:])
    per_col = (2 * u + u * u + 1e-5) * np.abs(emb_ref) + 6 * uh * np.concatenate([mag, mag], 1)
    dh = per_col @ np.abs(w.W1.astype(np.float64)).T
    return _second_layer(emb_ref, w, dh)


def within_half_bound(gpu, ref, emb_ref, w, mode):
    """max over events and outputs of |dflow| / (bound + 1e-6 (|flow| + 1e-3)); <= 1 passes."""
    b = acc16_flow_bound(emb_ref, w, mode) if mode & vk.ACC_FP16 else half_flow_bound(emb_ref, w, mode)
    d = np.abs(np.asarray(gpu, np.float64) - ref)
    return float(np.max(d / (b + 1e-6 * (np.abs(ref) + 1e-3))))


def flow_rel_err(gpu, ref, floor_frac=FLOW_FLOOR):
    gpu = np.asarray(gpu, np.float64)
    nr = np.linalg.norm(ref, axis=1)
    floor = floor_frac * np.median(nr)
    return np.linalg.norm(gpu - ref, axis=1) / np.maximum(nr, floor)
