"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never does, and there is no CPU fallback through it.

The arithmetic lives in ``veckm_oracle.c`` (plain C, FP64, OpenMP over output
events).  This module compiles it with gcc on first use and exposes it with
numpy arrays through ctypes.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariances, the agreement of the two encoder forms,
Lemma 1's density limit and hand-worked values.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "veckm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    P = C.c_void_p
    i64, i32, u32, f64 = C.c_int64, C.c_int32, C.c_uint32, C.c_double
    enc = [P, P, P, i64, u32, P, i64, i32, i32, i32, i32, i32, f64, P, P, P, P, P]
    for name in ("oracle_encode_direct", "oracle_encode_pooled"):
        fn = getattr(lib, name)
        fn.argtypes = enc
        fn.restype = C.c_int
    lib.oracle_mlp.argtypes = [P, i64, i32, i32, P, P, P, P, P]
    lib.oracle_mlp.restype = C.c_int
    lib.oracle_kde_query.argtypes = [P, i32, P, P, P, f64, f64, f64, P]
    lib.oracle_kde_query.restype = C.c_int
    lib.oracle_num_threads.restype = C.c_int
    lib.oracle_set_num_threads.argtypes = [C.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every oracle call to another build of veckm_oracle.c.

    Used by the mutation test, which compiles copies of the oracle with one
    planted mistake each and checks that the pins reject every copy.
    """
    global _lib
    _load()
    with _lock:
        old = _lib
        _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = old


SOURCE = _SRC


class OracleError(RuntimeError):
    pass


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def _encode(fn, x, y, t, t_ref, W, H, D, dx, dy, dt_us, T, X, Y, K=None):
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    n = x.shape[0]
    Karr = None if K is None else np.ascontiguousarray(K, dtype=np.int64)
    nK = n if Karr is None else Karr.shape[0]
    T = np.ascontiguousarray(T, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    emb = np.zeros((nK, 2 * D), dtype=np.float64)
    cnt = np.zeros(nK, dtype=np.int64)
    rc = fn(_ptr(x), _ptr(y), _ptr(t), n, int(t_ref), _ptr(Karr), nK, int(W), int(H), int(D),
            int(dx), int(dy), float(dt_us), _ptr(T), _ptr(X), _ptr(Y), _ptr(emb), _ptr(cnt))
    if rc != 0:
        raise OracleError(f"{fn.__name__} failed with status {rc}")
    return emb, cnt


def encode_direct(x, y, t, t_ref, W, H, D, dx, dy, dt_us, T, X, Y, K=None):
    """Eq. (emb), the O(N^2) adjacency form.  Returns (emb [nK, 2D] = [Re|Im], counts)."""
    return _encode(_load().oracle_encode_direct, x, y, t, t_ref, W, H, D, dx, dy, dt_us, T, X, Y, K)


def encode_pooled(x, y, t, t_ref, W, H, D, dx, dy, dt_us, T, X, Y, K=None):
    """Algorithm 1, the pooled form.  Returns (emb [nK, 2D] = [Re|Im], counts)."""
    return _encode(_load().oracle_encode_pooled, x, y, t, t_ref, W, H, D, dx, dy, dt_us, T, X, Y, K)


def mlp(emb, W1, b1, W2, b2):
    """flow = W2 ReLU(W1 emb + b1) + b2 in FP64 on FP32 weights.  emb: [nK, 2D]."""
    emb = np.ascontiguousarray(emb, dtype=np.float64)
    nK, in_dim = emb.shape
    D = in_dim // 2
    W1 = np.ascontiguousarray(W1, dtype=np.float32)
    hidden = W1.shape[0]
    b1 = np.ascontiguousarray(b1, dtype=np.float32)
    W2 = np.ascontiguousarray(W2, dtype=np.float32)
    b2 = np.ascontiguousarray(b2, dtype=np.float32)
    flow = np.zeros((nK, 2), dtype=np.float64)
    rc = _load().oracle_mlp(_ptr(emb), nK, D, hidden, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                            _ptr(flow))
    if rc != 0:
        raise OracleError(f"oracle_mlp failed with status {rc}")
    return flow


def kde_query(emb_row, T, X, Y, qt, qx, qy):
    """Lemma 1 read-back: Re((1/D) <emb, phi(q)>) at normalised offset (qt, qx, qy)."""
    e = np.ascontiguousarray(emb_row, dtype=np.float64)
    D = e.shape[0] // 2
    out = np.zeros(1, dtype=np.float64)
    rc = _load().oracle_kde_query(_ptr(e), D, _ptr(np.ascontiguousarray(T, dtype=np.float64)),
                                  _ptr(np.ascontiguousarray(X, dtype=np.float64)),
                                  _ptr(np.ascontiguousarray(Y, dtype=np.float64)),
                                  float(qt), float(qx), float(qy), _ptr(out))
    if rc != 0:
        raise OracleError(f"oracle_kde_query failed with status {rc}")
    return float(out[0])
