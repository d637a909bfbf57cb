"""Python binding of the C ABI in include/veckm.h (argument marshalling only).

Every step of the encoder and the flow head runs in the CUDA library
libveckm.so; this module only converts tensors to pointers and sizes and
passes the caller's CUDA stream.  PyTorch supplies device memory and streams.
There is no CPU fallback: if the library is missing or fails to load, the
import of this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

from . import build as _build

VECKM_OK, VECKM_EINVAL, VECKM_ENOMEM, VECKM_ECUDA = 0, -1, -2, -3
VECKM_ERANGE, VECKM_ETIMEOUT, VECKM_EBUSY, VECKM_EUNSUPPORTED = -4, -5, -6, -7
MLP_FP32, MLP_BF16, MLP_FP16 = 0, 1, 2
PATH_AUTO, PATH_DENSE, PATH_DIRECT = 0, 1, 2
ACC_FP16 = 4  # or-ed with MLP_BF16 / MLP_FP16: FP16 storage of the normalised pooled grid
STAGES = ("sort", "pixsum", "pool_rows", "counts", "pool_cols", "gather")

_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ERANGE", -5: "ETIMEOUT",
           -6: "EBUSY", -7: "EUNSUPPORTED"}


class VeckmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"veckm {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("D", C.c_int32),
                ("dx", C.c_int32), ("dy", C.c_int32), ("hidden", C.c_int32),
                ("dt_us", C.c_int64), ("t_span_us", C.c_int64), ("sigma2", C.c_double),
                ("freq_seed", C.c_uint64), ("h_T", C.c_void_p), ("h_X", C.c_void_p),
                ("h_Y", C.c_void_p), ("h_W1", C.c_void_p), ("h_b1", C.c_void_p),
                ("h_W2", C.c_void_p), ("h_b2", C.c_void_p), ("flags", C.c_uint32)]


class _ServerConfig(C.Structure):
    _fields_ = [("model", _Config), ("arena_bytes", C.c_int64), ("max_batch_packets", C.c_int32),
                ("max_batch_events", C.c_int64), ("batch_window_us", C.c_int32),
                ("window_us", C.c_int32), ("window_capacity", C.c_int64)]


class _Packet(C.Structure):
    _fields_ = [("stream_id", C.c_int32), ("tag", C.c_uint64), ("h_x", C.c_void_p),
                ("h_y", C.c_void_p), ("h_t", C.c_void_p), ("n", C.c_int64), ("t_ref_us", C.c_uint32),
                ("width", C.c_int32), ("height", C.c_int32), ("h_flow", C.c_void_p)]


class _Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("stream_id", C.c_int32), ("status", C.c_int),
                ("n", C.c_int64), ("latency_ms", C.c_double), ("batch_packets", C.c_int32)]


class _ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "admitted", "refused", "completed", "batches",
                                         "events_completed", "streams")] + \
               [(k, C.c_double) for k in ("p50_ms", "p99_ms", "max_ms", "wall_s", "gpu_busy_s")]


class _Slice(C.Structure):
    _fields_ = [("d_x", C.c_void_p), ("d_y", C.c_void_p), ("d_t", C.c_void_p), ("n", C.c_int64),
                ("t_ref_us", C.c_uint32), ("width", C.c_int32), ("height", C.c_int32)]


EXPORTS = ("veckm_create", "veckm_destroy", "veckm_encode", "veckm_encode_noalloc", "veckm_predict",
           "veckm_predict_host", "veckm_predict_host_async", "veckm_host_wait",
           "veckm_set_mlp_mode", "veckm_sync_status", "veckm_last_error",
           "veckm_get_frequencies", "veckm_set_timing", "veckm_stage_times",
           "veckm_last_launch_count", "veckm_canvas_layout", "veckm_predict_batch",
           "veckm_encode_batch", "veckm_plan_create", "veckm_plan_launch",
           "veckm_plan_kernel_count", "veckm_plan_destroy", "veckm_autotune",
           "veckm_server_create", "veckm_server_submit", "veckm_server_poll", "veckm_server_drain",
           "veckm_server_get_stats", "veckm_server_destroy", "veckm_kde_query", "veckm_set_path",
           "veckm_last_path", "veckm_set_path_model", "veckm_stream_create", "veckm_stream_push",
           "veckm_stream_window", "veckm_stream_accumulator", "veckm_stream_destroy",
           "veckm_set_wait_limit", "veckm_set_injection", "veckm_debug_fail_alloc",
           "veckm_debug_checks", "veckm_normals")
INJECT_NONE, INJECT_HEAD_STALL = 0, 1


def debug_fail_alloc(fail_at: int) -> int:
    """Counts the library's allocations from 0 again and fails allocation
    number fail_at (-1: none); returns the count since the previous call."""
    return int(lib().veckm_debug_fail_alloc(fail_at))


def debug_checks() -> Tuple[int, int]:
    """Bounds-checked build only: waits for the device and returns (number of
    indices that would have left their buffer since the previous call, where
    the first was: file number * 100000 + source line), then clears them."""
    n, line = C.c_int64(0), C.c_int32(0)
    _check(lib().veckm_debug_checks(C.byref(n), C.byref(line)))
    return int(n.value), int(line.value)


def library_path() -> str:
    return _build.CHECKED_LIB if os.environ.get("VECKM_LIBRARY") == "checked" else _build.LIB


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libveckm.so (building it first if needed) and declare its signatures.
    With VECKM_LIBRARY=checked in the environment, the bounds-checked build."""
    path = path or _build.build(checked=os.environ.get("VECKM_LIBRARY") == "checked")
    lib = C.CDLL(path)
    P, i64, u32, i32 = C.c_void_p, C.c_int64, C.c_uint32, C.c_int
    lib.veckm_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(_Config)]
    lib.veckm_destroy.argtypes = [P]
    lib.veckm_destroy.restype = None
    ev = [P, P, P, P, i64, u32, P, i64, P, P]
    lib.veckm_encode.argtypes = ev
    lib.veckm_encode_noalloc.argtypes = ev
    lib.veckm_encode_noalloc.restype = C.c_int
    lib.veckm_predict.argtypes = ev
    lib.veckm_predict_host.argtypes = ev
    lib.veckm_predict_host_async.argtypes = [P, P, P, P, i64, u32, P, i64, P,
                                             C.POINTER(C.c_int64)]
    lib.veckm_host_wait.argtypes = [P, i64]
    lib.veckm_set_mlp_mode.argtypes = [P, u32]
    lib.veckm_sync_status.argtypes = [P, P]
    lib.veckm_last_error.restype = C.c_char_p
    lib.veckm_get_frequencies.argtypes = [P, P, P, P]
    lib.veckm_set_timing.argtypes = [P, i32]
    lib.veckm_stage_times.argtypes = [P, P, P, i32]
    lib.veckm_last_launch_count.argtypes = [P]
    lib.veckm_set_wait_limit.argtypes = [P, i64]
    lib.veckm_set_injection.argtypes = [P, i32]
    lib.veckm_debug_fail_alloc.argtypes = [i64]
    lib.veckm_debug_fail_alloc.restype = i64
    lib.veckm_debug_checks.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    lib.veckm_debug_checks.restype = C.c_int
    lib.veckm_normals.argtypes = [C.c_uint64, i64, P]
    lib.veckm_normals.restype = None
    i32 = C.c_int32
    lib.veckm_canvas_layout.argtypes = [i32, P, P, i32, i32, i32, P, P, P, P]
    lib.veckm_predict_batch.argtypes = [P, P, i32, P, P]
    lib.veckm_encode_batch.argtypes = [P, P, i32, P, P]
    lib.veckm_plan_create.argtypes = [P, P, i32, P, i32, C.POINTER(C.c_void_p)]
    lib.veckm_plan_launch.argtypes = [P, P]
    lib.veckm_plan_kernel_count.argtypes = [P]
    lib.veckm_plan_destroy.argtypes = [P]
    lib.veckm_plan_destroy.restype = None
    lib.veckm_autotune.argtypes = [P, i32, i32, P, P]
    lib.veckm_server_create.argtypes = [C.POINTER(_ServerConfig), C.POINTER(C.c_void_p)]
    lib.veckm_server_submit.argtypes = [P, C.POINTER(_Packet)]
    lib.veckm_server_poll.argtypes = [P, P, i32, i32]
    lib.veckm_server_drain.argtypes = [P]
    lib.veckm_server_get_stats.argtypes = [P, C.POINTER(_ServerStats)]
    lib.veckm_server_destroy.argtypes = [P]
    lib.veckm_server_destroy.restype = None
    lib.veckm_kde_query.argtypes = [P, P, i64, P, P, P, P, i64, P, P]
    lib.veckm_set_path.argtypes = [P, i32]
    lib.veckm_last_path.argtypes = [P]
    lib.veckm_set_path_model.argtypes = [P, C.c_double, C.c_double, C.c_double]
    lib.veckm_stream_create.argtypes = [P, i64, i64, C.POINTER(C.c_void_p)]
    lib.veckm_stream_push.argtypes = [P, P, P, P, i64, C.c_uint32, P, i32, P]
    lib.veckm_stream_window.argtypes = [P, P, P]
    lib.veckm_stream_accumulator.argtypes = [P, P, P, P]
    lib.veckm_stream_destroy.argtypes = [P]
    lib.veckm_stream_destroy.restype = None
    for name in ("veckm_create", "veckm_encode", "veckm_predict", "veckm_predict_host",
                 "veckm_predict_host_async", "veckm_host_wait",
                 "veckm_set_mlp_mode", "veckm_sync_status", "veckm_get_frequencies",
                 "veckm_set_timing", "veckm_stage_times", "veckm_last_launch_count",
                 "veckm_canvas_layout", "veckm_predict_batch", "veckm_encode_batch",
                 "veckm_plan_create", "veckm_plan_launch", "veckm_plan_kernel_count",
                 "veckm_autotune", "veckm_server_create", "veckm_server_submit",
                 "veckm_server_poll", "veckm_server_drain", "veckm_server_get_stats",
                 "veckm_kde_query", "veckm_set_path", "veckm_last_path",
                 "veckm_set_path_model", "veckm_stream_create", "veckm_stream_push",
                 "veckm_stream_window", "veckm_stream_accumulator"):
        getattr(lib, name).restype = C.c_int
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status: int):
    if status != 0:
        raise VeckmError(status, lib().veckm_last_error().decode(errors="replace"))


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def normals(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, np.float64)
    lib().veckm_normals(C.c_uint64(seed), count, _np_ptr(out))
    return out


def canvas_layout(widths, heights, gap_x: int, gap_y: int, max_width: int):
    """Shelf packing of sensors on a canvas: (ox, oy, canvas_w, canvas_h)."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    h = np.ascontiguousarray(heights, dtype=np.int32)
    ox = np.zeros(w.size, np.int32)
    oy = np.zeros(w.size, np.int32)
    cw, ch = C.c_int32(), C.c_int32()
    _check(lib().veckm_canvas_layout(w.size, _np_ptr(w), _np_ptr(h), gap_x, gap_y, max_width,
                                     _np_ptr(ox), _np_ptr(oy), C.byref(cw), C.byref(ch)))
    return ox, oy, cw.value, ch.value


@dataclass
class Slice:
    """One slice of a batch: int16 x, y and int32 (uint32 bits) t CUDA tensors."""
    x: object
    y: object
    t: object
    t_ref: int
    width: int
    height: int

    @property
    def n(self) -> int:
        return int(self.x.numel())


def _slice_array(slices):
    arr = (_Slice * max(1, len(slices)))()
    for i, s in enumerate(slices):
        n = s.n
        arr[i] = _Slice(s.x.data_ptr() if n else None, s.y.data_ptr() if n else None,
                        s.t.data_ptr() if n else None, n, s.t_ref, s.width, s.height)
    return arr


class Plan:
    """A batch captured into a CUDA graph (veckm_plan_create); launch() replays it."""

    def __init__(self, enc, slices, out, predict: bool):
        self._keep = (slices, out)
        arr = _slice_array(slices)
        h = C.c_void_p()
        _check(lib().veckm_plan_create(enc.handle, arr, len(slices),
                                       C.c_void_p(out.data_ptr()) if out.numel() else None,
                                       1 if predict else 0, C.byref(h)))
        self._h = h
        self.out = out

    def launch(self, stream=None):
        _check(lib().veckm_plan_launch(self._h, Encoder._stream(stream)))
        return self.out

    @property
    def kernel_count(self) -> int:
        return int(lib().veckm_plan_kernel_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().veckm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Params:
    width: int
    height: int
    D: int = 64
    dx: int = 10
    dy: int = 10
    dt_us: int = 16_000
    t_span_us: int = 0
    hidden: int = 128
    sigma2: float = 25.0
    freq_seed: int = 0


def _make_config(p: Params, W1, b1, W2, b2, T, X, Y, flags: int, keep: list) -> _Config:
    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    cfg = _Config(width=p.width, height=p.height, D=p.D, dx=p.dx, dy=p.dy, hidden=p.hidden,
                  dt_us=p.dt_us, t_span_us=p.t_span_us, sigma2=p.sigma2,
                  freq_seed=p.freq_seed, flags=flags)
    for name, a, dt in (("h_T", T, np.float64), ("h_X", X, np.float64),
                        ("h_Y", Y, np.float64), ("h_W1", W1, np.float32),
                        ("h_b1", b1, np.float32), ("h_W2", W2, np.float32),
                        ("h_b2", b2, np.float32)):
        setattr(cfg, name, _np_ptr(arr(a, dt)))
    return cfg


def _host_ptr(a):
    """Address of a host buffer: a numpy array or a CPU torch tensor (pinned or not)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert not a.is_cuda and a.is_contiguous()
    return a.data_ptr()


class Server:
    """The native request loop (veckm_server_*): packets in, flows out.

    ``submit`` admits a packet (returns True) or refuses it when the device
    arena has no room (returns False).  Host buffers are kept referenced here
    until the packet's completion has been polled."""

    def __init__(self, p: Params, W1, b1, W2, b2, T=None, X=None, Y=None,
                 mlp_mode: int = MLP_FP32, arena_bytes: int = 0, max_batch_packets: int = 0,
                 max_batch_events: int = 0, batch_window_us: int = 0, window_us: int = 0,
                 window_capacity: int = 0):
        keep = []
        cfg = _ServerConfig(model=_make_config(p, W1, b1, W2, b2, T, X, Y, mlp_mode, keep),
                            arena_bytes=arena_bytes, max_batch_packets=max_batch_packets,
                            max_batch_events=max_batch_events, batch_window_us=batch_window_us,
                            window_us=window_us, window_capacity=window_capacity)
        h = C.c_void_p()
        _check(lib().veckm_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self.p = p
        self._bufs = {}
        self._next_tag = 1

    def submit(self, stream_id: int, x, y, t, t_ref: int, width: int, height: int, out,
               tag: Optional[int] = None) -> bool:
        if tag is None:
            tag = self._next_tag
            self._next_tag += 1
        n = int(x.shape[0])
        pk = _Packet(stream_id, tag, _host_ptr(x), _host_ptr(y), _host_ptr(t), n, t_ref, width,
                     height, _host_ptr(out))
        st = lib().veckm_server_submit(self._h, C.byref(pk))
        if st == VECKM_EBUSY:
            return False  # refused: no room in the arena (or for the stream's window)
        _check(st)
        self._bufs[tag] = (x, y, t, out)
        return True

    def poll(self, max_items: int = 1024, wait_ms: int = 0):
        arr = (_Completion * max_items)()
        k = lib().veckm_server_poll(self._h, arr, max_items, wait_ms)
        if k < 0:
            _check(k)
        out = []
        for i in range(k):
            c = arr[i]
            self._bufs.pop(c.tag, None)
            out.append({"tag": c.tag, "stream_id": c.stream_id, "status": c.status, "n": c.n,
                        "latency_ms": c.latency_ms, "batch_packets": c.batch_packets})
        return out

    def drain(self):
        _check(lib().veckm_server_drain(self._h))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().veckm_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().veckm_server_destroy(self._h)
            self._h = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """A sliding window over one sensor's events (veckm_stream_*), on an Encoder's context."""

    def __init__(self, enc, window_us: int, capacity: int):
        h = C.c_void_p()
        _check(lib().veckm_stream_create(enc.handle, window_us, capacity, C.byref(h)))
        self._h = h
        self.enc = enc

    def push(self, x, y, t, t_hi: int, out=None, predict: bool = True, stream=None):
        import torch
        n = x.numel()
        if out is None:
            out = torch.empty((n, 2 if predict else 2 * self.enc.p.D), dtype=torch.float32,
                              device="cuda")
        d = Encoder._dev
        _check(lib().veckm_stream_push(self._h, d(x, torch.int16), d(y, torch.int16),
                                       d(t, torch.int32), n, C.c_uint32(t_hi),
                                       d(out, torch.float32), 1 if predict else 0,
                                       Encoder._stream(stream)))
        return out

    def window_events(self, stream=None) -> int:
        v = C.c_int64()
        _check(lib().veckm_stream_window(self._h, C.byref(v), Encoder._stream(stream)))
        return v.value

    def accumulator(self, stream=None):
        p = self.enc.p
        acc = np.zeros((p.height, p.width, p.D // 2, 4), np.int64)
        cnt = np.zeros((p.height, p.width), np.int32)
        _check(lib().veckm_stream_accumulator(self._h, _np_ptr(acc), _np_ptr(cnt),
                                              Encoder._stream(stream)))
        return acc, cnt

    def close(self):
        if getattr(self, "_h", None):
            lib().veckm_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Encoder:
    """One veckm context: tables, weights and per-pixel accumulators on the GPU."""

    def __init__(self, p: Params, W1, b1, W2, b2, T=None, X=None, Y=None, mlp_mode: int = MLP_FP32):
        self.p = p
        keep = []
        cfg = _make_config(p, W1, b1, W2, b2, T, X, Y, mlp_mode, keep)
        h = C.c_void_p()
        _check(lib().veckm_create(C.byref(h), C.byref(cfg)))
        self._h = h
        self.mlp_mode = mlp_mode

    def close(self):
        if getattr(self, "_h", None):
            lib().veckm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_mlp_mode(self, mode: int):
        _check(lib().veckm_set_mlp_mode(self._h, mode))
        self.mlp_mode = mode

    def frequencies(self):
        D = self.p.D
        T, X, Y = (np.zeros(D), np.zeros(D), np.zeros(D))
        _check(lib().veckm_get_frequencies(self._h, _np_ptr(T), _np_ptr(X), _np_ptr(Y)))
        return T, X, Y

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    @staticmethod
    def _dev(t, dtype):
        if t is None:
            return None
        assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), (t.device, t.dtype)
        return C.c_void_p(t.data_ptr()) if t.numel() else None

    def _args(self, x, y, t, K):
        import torch
        n = x.numel()
        nK = n if K is None else K.numel()
        return (self._dev(x, torch.int16), self._dev(y, torch.int16), self._dev(t, torch.int32),
                n, self._dev(K, torch.int64), nK)

    def encode(self, x, y, t, t_ref: int, K=None, out=None, stream=None):
        """emb [nK, 2D] float32 on the device: [Re | Im] per requested event.

        x, y: int16 CUDA tensors; t: int32 CUDA tensor holding the uint32
        microsecond timestamps bit for bit; K: optional int64 CUDA tensor.
        """
        import torch
        xp, yp, tp, n, Kp, nK = self._args(x, y, t, K)
        if out is None:
            out = torch.empty((nK, 2 * self.p.D), dtype=torch.float32, device=x.device)
        _check(lib().veckm_encode(self._h, xp, yp, tp, n, C.c_uint32(t_ref), Kp, nK,
                                  self._dev(out, torch.float32), self._stream(stream)))
        return out

    def predict(self, x, y, t, t_ref: int, K=None, out=None, stream=None):
        """flow [nK, 2] float32 on the device."""
        import torch
        xp, yp, tp, n, Kp, nK = self._args(x, y, t, K)
        if out is None:
            out = torch.empty((nK, 2), dtype=torch.float32, device=x.device)
        _check(lib().veckm_predict(self._h, xp, yp, tp, n, C.c_uint32(t_ref), Kp, nK,
                                   self._dev(out, torch.float32), self._stream(stream)))
        return out

    def predict_host(self, x, y, t, t_ref: int, K=None, out=None, stream=None):
        """Host (CPU, ideally pinned) tensors in, host flows out; synchronising."""
        import torch
        n = x.numel()
        nK = n if K is None else K.numel()
        if out is None:
            out = torch.empty((nK, 2), dtype=torch.float32)

        def hp(a):
            return None if a is None or a.numel() == 0 else C.c_void_p(a.data_ptr())
        _check(lib().veckm_predict_host(self._h, hp(x), hp(y), hp(t), n, C.c_uint32(t_ref),
                                        hp(K), nK, hp(out), self._stream(stream)))
        return out

    def predict_host_async(self, x, y, t, t_ref: int, K=None, out=None) -> Tuple[int, object]:
        """Pipelined predict_host: returns (ticket, out) at once; out is filled
        after host_wait(ticket).  Inputs should be pinned CPU tensors; they
        are kept alive here until the call can no longer touch them."""
        import torch
        n = x.numel()
        nK = n if K is None else K.numel()
        if out is None:
            out = torch.empty((nK, 2), dtype=torch.float32, pin_memory=True)
        for a in (x, y, t, K, out):
            assert a is None or (not a.is_cuda and a.is_contiguous())

        def hp(a):
            return None if a is None or a.numel() == 0 else C.c_void_p(a.data_ptr())
        tk = C.c_int64(-1)
        _check(lib().veckm_predict_host_async(self._h, hp(x), hp(y), hp(t), n, C.c_uint32(t_ref),
                                              hp(K), nK, hp(out), C.byref(tk)))
        # issuing ticket k retired ticket k - 2 inside the library
        self._inflight = {k: v for k, v in getattr(self, "_inflight", {}).items()
                          if k >= tk.value - 1}
        self._inflight[tk.value] = (x, y, t, K, out)
        return tk.value, out

    def host_wait(self, ticket: int):
        """Block until the pipelined call `ticket` has finished; raise its error."""
        st = lib().veckm_host_wait(self._h, ticket)
        getattr(self, "_inflight", {}).pop(ticket, None)
        _check(st)

    def sync_status(self, stream=None):
        _check(lib().veckm_sync_status(self._h, self._stream(stream)))

    def set_timing(self, on: bool):
        _check(lib().veckm_set_timing(self._h, 1 if on else 0))

    def stage_times(self):
        """(milliseconds per stage summed over timed calls, number of timed calls)."""
        ms = np.zeros(len(STAGES), np.float64)
        calls = np.zeros(len(STAGES), np.int64)
        _check(lib().veckm_stage_times(self._h, _np_ptr(ms), _np_ptr(calls), len(STAGES)))
        return dict(zip(STAGES, ms)), dict(zip(STAGES, calls))

    def last_launch_count(self) -> int:
        return int(lib().veckm_last_launch_count(self._h))

    def predict_batch(self, slices, out=None, stream=None):
        """Flows [sum n, 2] of every event of every slice (slice order)."""
        import torch
        N = sum(s.n for s in slices)
        if out is None:
            out = torch.empty((N, 2), dtype=torch.float32, device="cuda")
        arr = _slice_array(slices)
        _check(lib().veckm_predict_batch(self._h, arr, len(slices),
                                         C.c_void_p(out.data_ptr()) if N else None,
                                         self._stream(stream)))
        return out

    def encode_batch(self, slices, out=None, stream=None):
        """Encodings [sum n, 2D] of every event of every slice (slice order)."""
        import torch
        N = sum(s.n for s in slices)
        if out is None:
            out = torch.empty((N, 2 * self.p.D), dtype=torch.float32, device="cuda")
        arr = _slice_array(slices)
        _check(lib().veckm_encode_batch(self._h, arr, len(slices),
                                        C.c_void_p(out.data_ptr()) if N else None,
                                        self._stream(stream)))
        return out

    def plan(self, slices, out=None, predict: bool = True) -> Plan:
        import torch
        N = sum(s.n for s in slices)
        if out is None:
            out = torch.empty((N, 2 if predict else 2 * self.p.D), dtype=torch.float32,
                              device="cuda")
        return Plan(self, slices, out, predict)

    def set_path(self, path: int):
        _check(lib().veckm_set_path(self._h, path))

    def set_wait_limit(self, cycles: int):
        _check(lib().veckm_set_wait_limit(self._h, cycles))

    def set_injection(self, what: int):
        _check(lib().veckm_set_injection(self._h, what))

    def last_path(self) -> int:
        return int(lib().veckm_last_path(self._h))

    def set_path_model(self, pixel_ns: float, flow_dense_ns: float, flow_window_ns: float):
        _check(lib().veckm_set_path_model(self._h, pixel_ns, flow_dense_ns, flow_window_ns))

    def kde_query(self, emb, rows, qt, qx, qy, out=None, stream=None):
        """Lemma 1 read-back at integer offsets (qt us, qx, qy px) from the events of emb rows."""
        import torch
        nq = rows.numel()
        if out is None:
            out = torch.empty(nq, dtype=torch.float32, device=emb.device)
        _check(lib().veckm_kde_query(self._h, self._dev(emb, torch.float32), emb.shape[0],
                                     self._dev(rows, torch.int64), self._dev(qt, torch.int32),
                                     self._dev(qx, torch.int32), self._dev(qy, torch.int32), nq,
                                     self._dev(out, torch.float32), self._stream(stream)))
        return out

    def autotune(self, width: int, height: int, stream=None):
        """Pooling launch shapes chosen for width x height: (rows seg, rows warps, cols seg, cols warps)."""
        t = np.zeros(4, np.int32)
        _check(lib().veckm_autotune(self._h, width, height, self._stream(stream), _np_ptr(t)))
        return tuple(int(v) for v in t)
