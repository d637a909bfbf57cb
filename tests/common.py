"""Helpers shared by the GPU tests: build a context from seeded inputs, move a
slice to the device, and the error measures the parity bars are stated in."""
import numpy as np

from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk

# Parity bars (derivations in the design notes):
#  - FP32 encoder: per requested event, ||emb_gpu - emb_ref||_2 / ||emb_ref||_2.
#  - flows: per event ||flow_gpu - flow_ref||_2 / max(||flow_ref||_2, floor) with
#    floor = FLOW_FLOOR * median ||flow_ref||_2.
EMB_TOL_FP32 = 1e-4
FLOW_TOL_FP32 = 1e-4
FLOW_TOL = {vk.MLP_FP32: 1e-4}
FLOW_FLOOR = 1e-3
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


def half_flow_bound(emb_ref, w, mode):
    """A-priori bound on |flow_gpu - flow_ref| per output for a first layer whose
    operands (emb and W1) are rounded to BF16/FP16 (unit roundoff u) and whose
    products are accumulated in FP32:
        |dflow_o| <= sum_j |W2_oj| * (2u + u^2 + 1e-5) * sum_c |W1_jc e_c|
    (each rounded product is W e (1 + d1)(1 + d2); ReLU is 1-Lipschitz; the
    1e-5 covers FP32 accumulation over at most 256 terms and the FP32 error
    of the encoder)."""
    u = UNIT_ROUNDOFF[mode]
    a = np.abs(emb_ref) @ np.abs(w.W1.astype(np.float64)).T          # [nK, hidden]
    return (2 * u + u * u + 1e-5) * (a @ np.abs(w.W2.astype(np.float64)).T)  # [nK, 2]


def acc16_flow_bound(emb_ref, w, mode):
    """Bound for the FP16 pooled grid (VECKM_ACC_FP16) on top of the MMA operand
    rounding: the stored normalised pooled value p and the phase are each
    rounded once to FP16 (u_h = 2^-11) and the packed half2 product
    Re = p_r c + p_i s, Im = p_i c - p_r s adds a rounding per multiply and per
    fused add, so |d e_c| <= 4 u_h (|p_r| + |p_i|) <= 4 sqrt(2) u_h |p_d| < 6 u_h |e_d|
    for both columns c of channel d (|p_d| = |e_d|, the phase has modulus 1).
        |dflow_o| <= sum_j |W2_oj| sum_c |W1_jc| (2 u |e_c| + 6 u_h |e_d(c)| + 1e-5 |e_c|)"""
    u = UNIT_ROUNDOFF[mode & 3]
    uh = 2.0 ** -11
    D = emb_ref.shape[1] // 2
    mag = np.hypot(emb_ref[:, :D], emb_ref[:, D:])
    per_col = (2 * u + u * u + 1e-5) * np.abs(emb_ref) + 6 * uh * np.concatenate([mag, mag], 1)
    a = per_col @ np.abs(w.W1.astype(np.float64)).T
    return a @ np.abs(w.W2.astype(np.float64)).T


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
