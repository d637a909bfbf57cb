"""Benchmark: normal flows per second of the encoder + flow head on one slice.

One step = one veckm_predict over the whole slice (every event is a requested
flow): sort by pixel, per-pixel phase sums, two pooling passes, window counts,
gather fused with the perceptron.  Inputs are resident in HBM when the timed region starts; the
accumulators written by every step (2 x 157 MB at 640x480, D=64) exceed the
129 MB L2, so no explicit flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--mode bf16|fp16|fp32] [--lean]

Prints one JSON line (rank 0).  With --impl reference the same metric is
measured for the FP64 CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "normal flows/sec on 1 GB300 (chosen vs plain FP32) at stated err vs FP64; p50/p99 ms"
UNIT = "flows/s"
DEFAULT_WORKLOAD = "slice-640x480-2M"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "bf16_tflops": float(pk["bf16_tflops"]),
                "bf16_tflops_sustained": float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


class _NvmlPoller:
    """SM clock and clock-event reasons read through NVML (the driver's
    library, loaded with ctypes; read-only queries) every millisecond from a
    thread, so that a timed region of a few milliseconds still gets samples.
    Reason bits are NVML's public clock-event reason flags."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, device: int):
        import ctypes as C
        self.C = C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        import torch
        want = str(torch.cuda.get_device_properties(device).uuid).lower().replace("gpu-", "")
        count = C.c_uint()
        if lib.nvmlDeviceGetCount_v2(C.byref(count)) != 0:
            raise RuntimeError("nvmlDeviceGetCount failed")
        handles = []
        for i in range(count.value):
            h, buf = C.c_void_p(), C.create_string_buffer(96)
            if lib.nvmlDeviceGetHandleByIndex_v2(i, C.byref(h)) != 0:
                continue
            if lib.nvmlDeviceGetUUID(h, buf, 96) != 0:
                continue
            handles.append((buf.value.decode("ascii").lower().replace("gpu-", ""), h))
        match = [h for u, h in handles if u == want]
        if not match and len(handles) == 1:
            match = [handles[0][1]]
        if not match:
            raise RuntimeError("no NVML device with the CUDA device's UUID")
        self.h = match[0]
        self.lib = lib
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        mx = C.c_uint()
        self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(self.h, 1, C.byref(mx)) == 0 \
            else None
        self.samples, self.flags = [], 0
        self.run = False

    def _loop(self):
        C = self.C
        mhz, rs = C.c_uint(), C.c_ulonglong()
        while self.run:
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, C.byref(mhz)) == 0:  # 1: SM clock
                self.samples.append(float(mhz.value))
            if self.reasons_fn(self.h, C.byref(rs)) == 0:
                self.flags |= int(rs.value)
            time.sleep(0.001)

    def start(self):
        self.run = True
        self.th = threading.Thread(target=self._loop, daemon=True)
        self.th.start()

    def stop(self):
        self.run = False
        self.th.join(timeout=2)
        if not self.samples:
            return None
        return {"sm_mhz": float(np.median(self.samples)), "sm_max_mhz": self.max_mhz,
                "samples": len(self.samples), "source": "nvml, 1 ms polling",
                "reasons": sorted(v for k, v in self.REASONS.items() if self.flags & k)}


class ClockSampler:
    """Clock and throttle samples while the timed region runs: NVML polled
    in-process when the driver's library loads, else nvidia-smi."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.nvml = None
        self.lines = []

    def start(self):
        self.nvml = None
        try:
            self.nvml = _NvmlPoller(self.index)
            self.nvml.start()
            return
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            r = self.nvml.stop()
            if r is not None:
                return r
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def _oracle_single_thread(oracle, sl, D, T, X, Y, w, K):
    """The same oracle call on one host thread (a smaller sample), beside the
    all-core figure; None if it cannot be timed."""
    cores = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        t0 = time.perf_counter()
        emb, _ = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D,
                                      10, 10, 16_000.0, T, X, Y, K=K)
        oracle.mlp(emb, w.W1, w.b1, w.W2, w.b2)
        dt = time.perf_counter() - t0
        return {"value": len(K) / dt, "unit": UNIT, "cores": 1,
                "sample": f"{len(K)} of the same requested events, {dt:.1f} s"}
    except Exception:
        return None
    finally:
        oracle.set_num_threads(cores)


# The sources a stage's DRAM traffic depends on: the translation unit of its
# kernels, plus the pipeline that launches them and the headers they share.
_COMMON_SRC = ("veckm.cu", "ctx.h", "veckm_internal.h", "chain.cuh", "check.cuh", "phase.cuh")
_STAGE_SRC = {"gather": "mlp_tc.cu", "sort": "kernels.cu", "pixsum": "kernels.cu",
              "pool_rows": "kernels.cu", "pool_cols": "kernels.cu", "counts": "kernels.cu"}


def stage_digest(name: str) -> str:
    """Hash of the sources the stage's kernels are built and launched from."""
    src = os.path.join(ROOT, "paper_2504_19417_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted((_STAGE_SRC[name],) + _COMMON_SRC):
        with open(os.path.join(src, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _kernel_traffic(name: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the stage's
    sources are unchanged since the capture (their hash recorded beside it)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path) or name not in _STAGE_SRC:
        return None
    digest = stage_digest(name)
    for ln in open(path):
        f = ln.split()
        if len(f) >= 4 and not ln.startswith("#") and f[0] == name and f[1] == workload:
            return float(f[2]) if f[3] == digest else None
    return None


def source_digest() -> str:
    src = os.path.join(ROOT, "paper_2504_19417_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted(os.listdir(src)):
        if fn.endswith((".cu", ".h", ".cuh")):
            with open(os.path.join(src, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def algorithmic_bytes(sl, D, nK, touched, touched_K, acc16=False):
    """Bytes each stage must move at minimum (one launch), per the model in the
    design notes: complex FP32 = 8 B per channel, counts and offsets 4 B,
    events 8 B (x, y int16 + t uint32), sorted records 12 B (t, index, pixel),
    flows 8 B."""
    P = sl.width * sl.height
    pix = 8 * D
    N = sl.n
    return {
        "sort": 8 * N + 12 * N + 16 * P,
        "pixsum": 8 * N + 4 * P + P * pix,
        "pool_rows": 2 * P * pix,
        "pool_cols": P * pix + (P * pix // 2 if acc16 else P * pix),
        "counts": 16 * P,
        "gather": 12 * nK + touched_K * (pix // 2 if acc16 else pix + 4) + 8 * nK,
    }


def mlp_flops(nK, D, hidden=128):
    return 2.0 * nK * (2 * D * hidden + 2 * hidden)


def _dist():
    """(module, rank, world size, local rank); one process per GPU under
    torchrun.  VECKM_DIST_BACKEND selects the backend (nccl by default; the
    CPU tests use gloo)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(os.environ.get("VECKM_DIST_BACKEND", "nccl"))
        return dist, int(os.environ["RANK"]), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def max_over_ranks(dist, x: float) -> float:
    """The largest x over all ranks (the job takes as long as its slowest rank)."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_slice_def(workload: str, rank: int, scale: float = 1.0) -> dict:
    """The generator arguments of this rank's slice: the workload's shape with
    a seed of its own (weak scaling: every rank encodes an independent slice)."""
    from paper_2504_19417_gb300 import synth
    w = dict(synth.WORKLOADS[workload])
    w["seed"] = w["seed"] + 100 * rank
    w["n"] = max(1, int(round(w["n"] * scale)))
    return w


def job_rate(ws: int, units_per_rank: float, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the max time."""
    return ws * units_per_rank * steps / (total_ms / 1000.0)


def run_reference(args):
    """The FP64 CPU oracle as it stands, on bounded samples of the workload."""
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2504_19417_gb300 import synth
    sl, D = synth.workload(args.workload)
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    rng = np.random.default_rng(7)
    S = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        K = np.sort(rng.choice(sl.n, S, replace=False)).astype(np.int64)
        t0 = time.perf_counter()
        emb, _ = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                      16_000.0, T, X, Y, K=K)
        oracle.mlp(emb, w.W1, w.b1, w.W2, w.b2)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = S * len(times) / tot
    cores = oracle.num_threads()
    sample = (f"{S} requested events per step (random, all {sl.n} slice events scattered), "
              f"FP64 pooled form of Algorithm 1 + perceptron, OpenMP over requested events")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "D": D, "window": "21x21"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch
    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    modes = {"bf16": vk.MLP_BF16, "fp16": vk.MLP_FP16, "fp32": vk.MLP_FP32,
             "fp16-acc16": vk.MLP_FP16 | vk.ACC_FP16, "bf16-acc16": vk.MLP_BF16 | vk.ACC_FP16}
    mode = modes[args.mode]
    w_def = rank_slice_def(args.workload, rank, args.scale)
    D = w_def.pop("D")
    sl = synth.event_slice(**w_def)
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    span = int(sl.t.max()) - sl.t_ref
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=10, dy=10, dt_us=16_000,
                  t_span_us=span)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    tuned = enc.autotune(sl.width, sl.height) if not args.no_autotune else None
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    nK = sl.n
    flow = torch.empty((nK, 2), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)

    def timed(nsteps, per_step=True):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        evs[0].record(stream)
        for i in range(nsteps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
        per = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(nsteps)])
        total_ms = max_over_ranks(dist, float(evs[0].elapsed_time(evs[-1])))
        return total_ms, per, wall

    clocks = ClockSampler(local)
    if not args.lean:
        clocks.start()
    total_ms, per, wall = timed(args.steps)
    launches_per_step = enc.last_launch_count()
    clk = clocks.stop() if not args.lean else None
    # Stage times: a second timed pass of the same steps with the library's
    # per-stage event marks on.  With the marks on, the library launches each
    # stage after a mark in full order instead of chained to the kernel before
    # it, so the step above is timed without them.
    stage_ms, stage_calls = {}, {}
    if not args.lean:
        enc.set_timing(True)
        timed(args.steps)
        stage_ms, stage_calls = enc.stage_times()
        enc.set_timing(False)
    enc.sync_status()
    value = job_rate(ws, nK, args.steps, total_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "f32+bf16", "fp16": "f32+f16", "fp32": "f32",
                  "fp16-acc16": "f32+f16", "bf16-acc16": "f32+f16+bf16"}[args.mode],
        "data": "synthetic",
        "config": {"workload": args.workload, "sensor": f"{sl.width}x{sl.height}",
                   "events_per_slice": sl.n, "flows_per_step": nK, "D": D, "window": "21x21",
                   "dt_us": 16_000, "mlp": f"{2 * D}->128->2 ReLU", "mlp_precision": args.mode,
                   "parallelism": f"replicas x{ws}, one slice per GPU",
                   "pooling_shapes": ({"rows_seg": tuned[0], "rows_warps": tuned[1],
                                       "cols_seg": tuned[2], "cols_warps": tuned[3]}
                                      if tuned else "default"),
                   "l2": "inputs larger than L2 (each step writes 2 x accumulator grid)"},
        "gpu_launches": int(launches_per_step * args.steps),
    }
    if args.lean:
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out["clocks"] = clk
    # per-kernel roofline from CUDA events recorded on the launching stream
    pk = _peaks()
    key = sl.y.astype(np.int64) * sl.width + sl.x
    touched = int(np.unique(key).size)
    ab = algorithmic_bytes(sl, D, nK, touched, touched, acc16=bool(mode & vk.ACC_FP16))
    kern = {}
    for name in stage_ms:
        n = max(1, int(stage_calls[name]))
        ms = stage_ms[name] / n
        kern[name] = {"ms": ms, "GB/s": ab[name] / (ms * 1e-3) / 1e9 if ms > 0 else None,
                      "bytes": ab[name]}
    # the window counts run on a side stream under the sort, the pixel sums
    # and the row pass: their stage time is what the join still waits
    kern["counts"]["GB/s"] = None
    kern["counts"]["note"] = "side stream, overlapped; ms = residual wait at the join"
    kern["gather"]["TFLOP/s"] = mlp_flops(nK, D) / (kern["gather"]["ms"] * 1e-3) / 1e12
    dom = max(kern, key=lambda k: kern[k]["ms"])
    kd = kern[dom]
    if dom == "gather" and mode != vk.MLP_FP32 and \
            kd["TFLOP/s"] / pk["bf16_tflops_sustained"] > kd["GB/s"] / pk["hbm_gbs"]:
        roof = {"bound": "tensor", "achieved": kd["TFLOP/s"], "peak": pk["bf16_tflops_sustained"],
                "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": kd["GB/s"], "peak": pk["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom
    roof["timing"] = ("CUDA events on the launching stream around each stage, a second timed "
                      "pass of the same steps with the stage marks on")
    roof["peak_source"] = pk["source"]
    tr = _kernel_traffic(dom, args.workload)
    roof["traffic"] = tr
    roof["algorithmic_bytes"] = kd["bytes"]
    out["roofline"] = roof
    out["kernels"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                          for kk, vv in v.items()} for k, v in kern.items()}
    encoder_ms = sum(kern[k]["ms"] for k in kern if k != "gather")
    # the survey's per-stage model: events read once (9 B each), the
    # per-pixel accumulator (8D + 4 B) written once and read and written once
    # by the pooling
    P = sl.width * sl.height
    survey_bytes = 9 * sl.n + 3 * P * (8 * D + 4)
    out["encoder_roofline"] = {
        "algorithmic_bytes": int(sum(ab[k] for k in ab if k != "gather")),
        "ms": encoder_ms,
        "frac_of_hbm": (sum(ab[k] for k in ab if k != "gather") / (encoder_ms * 1e-3) / 1e9)
        / pk["hbm_gbs"] if encoder_ms > 0 else None,
        "survey_model_bytes": int(survey_bytes),
        "survey_model_frac": (survey_bytes / (encoder_ms * 1e-3) / 1e9) / pk["hbm_gbs"]
        if encoder_ms > 0 else None}

    # plain FP32 form on the same slice and GPU
    if mode != vk.MLP_FP32:
        enc.set_mlp_mode(vk.MLP_FP32)
        pms, pper, _ = timed(max(3, args.steps // 2))
        out["plain_fp32"] = {"value": ws * nK * len(pper) / (pms / 1000.0),
                             "ms_per_step": pms / len(pper),
                             "p50_ms": float(np.percentile(pper, 50)),
                             "p99_ms": float(np.percentile(pper, 99))}
        enc.set_mlp_mode(mode)

    # end to end through the public host-buffer entry points (pinned memory):
    # the pipelined call, two in flight (step k+1's upload and step k-1's
    # download overlap step k's computation), with two host buffer sets as an
    # application alternating between packets would hold; the synchronous
    # call is reported beside it
    bufs = []
    for _ in range(2):
        bufs.append((torch.from_numpy(sl.x).pin_memory(), torch.from_numpy(sl.y).pin_memory(),
                     torch.from_numpy(sl.t.view(np.int32)).pin_memory(),
                     torch.empty((nK, 2), dtype=torch.float32).pin_memory()))

    def pipelined(steps):
        prev = None
        for k in range(steps):
            hx, hy, ht, hf = bufs[k & 1]
            tk, _ = enc.predict_host_async(hx, hy, ht, sl.t_ref, out=hf)
            if prev is not None:
                enc.host_wait(prev)
            prev = tk
        enc.host_wait(prev)

    pipelined(3)
    ne = max(3, args.steps // 2)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    pipelined(ne)
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    out["e2e"] = {"value": ws * nK * ne / e2e_s, "unit": UNIT, "h2d_bytes_per_step": sl.n * 8,
                  "d2h_bytes_per_step": nK * 8, "ms_per_step": 1000 * e2e_s / ne,
                  "api": "veckm_predict_host_async + veckm_host_wait, 2 in flight"}
    hx, hy, ht, hflow = bufs[0]
    for _ in range(2):
        enc.predict_host(hx, hy, ht, sl.t_ref, out=hflow, stream=stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(ne):
        enc.predict_host(hx, hy, ht, sl.t_ref, out=hflow, stream=stream)
    sync_s = max_over_ranks(dist, time.perf_counter() - t0)
    out["e2e_sync"] = {"value": ws * nK * ne / sync_s, "unit": UNIT,
                       "ms_per_step": 1000 * sync_s / ne, "api": "veckm_predict_host"}

    # CPU baseline: the FP64 oracle on a bounded sample, rank 0 at N=1 only;
    # the same sample gives the per-output error of this run against FP64.
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(7)
        S = args.cpu_sample
        K = np.sort(rng.choice(sl.n, S, replace=False)).astype(np.int64)
        t0 = time.perf_counter()
        emb_ref, _ = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D,
                                          10, 10, 16_000.0, T, X, Y, K=K)
        flow_ref = oracle.mlp(emb_ref, w.W1, w.b1, w.W2, w.b2)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {
            "value": S / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{S} random requested events of the {sl.n}-event slice (all events "
                      f"scattered), FP64 pooled form + perceptron, {dt:.1f} s"}
        single = _oracle_single_thread(oracle, sl, D, T, X, Y, w, K[: max(1, S // 10)])
        if single:
            out["cpu_baseline"]["single_thread"] = single
        Kd = torch.from_numpy(K).cuda()
        emb_g = enc.encode(x, y, t, sl.t_ref, K=Kd).cpu().numpy().astype(np.float64)
        flow_g = enc.predict(x, y, t, sl.t_ref, K=Kd).cpu().numpy().astype(np.float64)
        e_err = np.linalg.norm(emb_g - emb_ref, axis=1) / np.linalg.norm(emb_ref, axis=1)
        nr = np.linalg.norm(flow_ref, axis=1)
        f_err = np.linalg.norm(flow_g - flow_ref, axis=1) / np.maximum(nr, 0.25 * np.median(nr))
        f_abs = np.abs(flow_g - flow_ref)
        out["err_vs_fp64"] = {
            "sample": S, "emb_rel_l2_max": float(e_err.max()), "emb_rel_l2_mean": float(e_err.mean()),
            "flow_rel_max": float(f_err.max()), "flow_rel_mean": float(f_err.mean()),
            "flow_abs_max": float(f_abs.max()), "flow_abs_mean": float(f_abs.mean()),
            "flow_rel_floor": "0.25 x median |flow|"}
    if rank == 0 and not args.no_stream:
        try:
            out["stream"] = stream_leg(args, mode, stream)
        except Exception as e:  # the headline line is printed regardless
            out["stream"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_small:
        try:
            out["small_slice"] = small_leg(args, mode, stream)
        except Exception as e:  # the headline line is printed regardless
            out["small_slice"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_sparse:
        try:
            out["sparse_k"] = sparse_leg(args, mode, stream)
        except Exception as e:  # the headline line is printed regardless
            out["sparse_k"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_precision:
        try:
            out["precision"] = precision_leg(args, stream)
        except Exception as e:  # the headline line is printed regardless
            out["precision"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_recipes:
        try:
            out["recipes"] = recipes_leg(args, mode, stream)
        except Exception as e:  # the headline line is printed regardless
            out["recipes"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_batch:
        try:
            out["batch"] = batch_leg(args, mode, stream)
        except Exception as e:  # the headline line is printed regardless
            out["batch"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_serving:
        try:
            out["serving"] = serving_windows_leg(args, mode)
        except Exception as e:  # the headline line is printed regardless
            out["serving"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            out["serving"]["packets_as_slices"] = serving_leg(args, mode)
        except Exception as e:
            out["serving"]["packets_as_slices"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out), flush=True)


def stream_leg(args, mode, stream):
    """Sliding window: the 640x480 slice (2 M events over 50 ms) replayed as a
    stream of 2 ms packets into a 32 ms window (2 delta_t) whose per-pixel sums
    stay resident; each push adds the packet, expires what left and predicts
    the packet's flows.  Per-push device time (CUDA events) and throughput."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    sl, D = synth.workload("slice-640x480-2M")
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=10, dy=10, dt_us=16_000,
                  t_span_us=32_000)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    enc.autotune(sl.width, sl.height, stream)
    st = vk.Stream(enc, 32_000, sl.n)
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    bounds = np.arange(int(sl.t[0]), int(sl.t[-1]) + 2_001, 2_000)
    cuts = np.searchsorted(sl.t, bounds, side="left")
    out = torch.empty((sl.n, 2), dtype=torch.float32, device="cuda")
    evs, sizes = [], []
    for q in range(len(bounds) - 1):
        i, j = int(cuts[q]), int(cuts[q + 1])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.push(x[i:j], y[i:j], t[i:j], int(bounds[q + 1]) - 1, out=out[i:j], stream=stream)
        b.record(stream)
        evs.append((a, b))
        sizes.append(j - i)
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    enc.sync_status()
    steady = ms[16:]  # after the window has filled (32 ms = 16 packets)
    n_steady = int(np.sum(sizes[16:]))
    res = {"workload": "640x480 slice (2 M events, 50 ms) as 2 ms packets, 32 ms window",
           "packets": len(ms), "mean_events_per_packet": float(np.mean(sizes)),
           "window_events_at_end": st.window_events(),
           "push_ms_p50": float(np.percentile(steady, 50)),
           "push_ms_p99": float(np.percentile(steady, 99)),
           "flows_per_s": n_steady / (float(steady.sum()) * 1e-3), "unit": UNIT,
           "resident": "64-bit fixed-point per-pixel sums (exact add/expire) + counts"}
    st.close()
    enc.close()
    return res


def small_leg(args, mode, stream):
    """The small single-slice case: 346x260, 20,000 events over 10 ms (D = 64,
    21x21 window), every event requested; the chosen mode and the plain FP32
    form, per call with the inputs resident (the mean over back-to-back calls;
    p50 and p99 from a second pass with an event after each call),
    the chosen mode also as a one-slice captured plan, and the flows' error
    against the FP64 oracle on every event."""
    import torch
    import oracle
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    sl, D = synth.workload("slice-346x260-20k")
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=10, dy=10, dt_us=16_000,
                  t_span_us=int(sl.t.max()) - sl.t_ref)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    enc.autotune(sl.width, sl.height, stream)
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    flow = torch.empty((sl.n, 2), dtype=torch.float32, device="cuda")
    e = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10, 16_000.0,
                             T, X, Y)[0]
    fref = oracle.mlp(e, w.W1, w.b1, w.W2, w.b2)
    nref = np.linalg.norm(fref, axis=1)
    floor = 0.25 * np.median(nref)
    res = {"workload": f"slice-346x260-20k ({sl.n} events, 10 ms, D={D}, 21x21)"}
    for name, m in ((args.mode, mode), ("fp32", vk.MLP_FP32)):
        enc.set_mlp_mode(m)
        for _ in range(args.warmup):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        k = max(10, args.steps)
        # the mean over back-to-back calls (two events around all of them),
        # then p50/p99 from an event after each call
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for i in range(k):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        b.record(stream)
        b.synchronize()
        mean_ms = a.elapsed_time(b) / k
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(k):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
            evs[i + 1].record(stream)
        evs[-1].synchronize()
        per = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(k)])
        f = flow.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(f - fref, axis=1) / np.maximum(nref, floor)
        res[name] = {"flows_per_s": sl.n / (mean_ms * 1e-3),
                     "ms_per_call": mean_ms, "p50_ms": float(np.percentile(per, 50)),
                     "p99_ms": float(np.percentile(per, 99)),
                     "kernels_per_call": enc.last_launch_count(),
                     "flow_rel_max": float(rel.max()), "flow_rel_mean": float(rel.mean()),
                     "flow_rel_floor": "0.25 x median |flow|"}
    # the same slice as a one-slice plan: the whole call captured in a CUDA
    # graph and replayed (launch overhead paid once per replay, not per kernel)
    enc.set_mlp_mode(mode)
    plan = enc.plan([vk.Slice(x, y, t, sl.t_ref, sl.width, sl.height)], out=flow)
    for _ in range(args.warmup):
        plan.launch(stream)
    k = max(10, args.steps)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for i in range(k):
        plan.launch(stream)
    b.record(stream)
    b.synchronize()
    mean_ms = a.elapsed_time(b) / k
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(k):
        plan.launch(stream)
        evs[i + 1].record(stream)
    evs[-1].synchronize()
    per = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(k)])
    f = flow.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(f - fref, axis=1) / np.maximum(nref, floor)
    res[args.mode + "_plan"] = {"flows_per_s": sl.n / (mean_ms * 1e-3),
                                "ms_per_call": mean_ms,
                                "p50_ms": float(np.percentile(per, 50)),
                                "p99_ms": float(np.percentile(per, 99)),
                                "kernels_per_call": plan.kernel_count,
                                "flow_rel_max": float(rel.max())}
    plan.close()
    enc.sync_status()
    enc.close()
    return res


def sparse_leg(args, mode, stream):
    """The paper's runtime example (Section 3): 0.5 M events and 10 k requested
    flows with a 17x17 window (dx = dy = 8), here on the 640x480 slice: the
    dense pooled form, the direct window form and the runtime-model choice.
    Also the model's coefficients measured on this run (ns)."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    sl, D = synth.workload("slice-640x480-2M", scale=0.25)
    r = synth.RECIPES["640x480_32ms_C64_k8"]
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=r["dx"], dy=r["dy"], dt_us=r["dt_us"],
                  t_span_us=int(sl.t.max()) - sl.t_ref)
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    enc.autotune(sl.width, sl.height, stream)
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    rng = np.random.default_rng(9)
    nK = 10_000
    K = torch.from_numpy(np.sort(rng.choice(sl.n, nK, replace=False)).astype(np.int64)).cuda()
    flow = torch.empty((nK, 2), dtype=torch.float32, device="cuda")
    res = {"workload": f"640x480, {sl.n} events, {nK} requested flows, 17x17 window"}
    stages = {}
    for name, path in (("dense", vk.PATH_DENSE), ("direct", vk.PATH_DIRECT), ("auto", vk.PATH_AUTO)):
        enc.set_path(path)
        for _ in range(args.warmup):
            enc.predict(x, y, t, sl.t_ref, K=K, out=flow, stream=stream)
        k = max(3, args.steps // 2)
        # the calls timed without the stage marks, then again with them for
        # the stage times (with the marks on, stages launch in full order)
        for timing in (False, True):
            enc.set_timing(timing)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                enc.predict(x, y, t, sl.t_ref, K=K, out=flow, stream=stream)
            b.record(stream)
            b.synchronize()
            if not timing:
                ms = a.elapsed_time(b) / k
        st, calls = enc.stage_times()
        enc.set_timing(False)
        stages[name] = {s_: 1000 * v / max(1, calls[s_]) for s_, v in st.items()}
        res[name] = {"ms_per_call": ms, "flows_per_s": nK / (ms * 1e-3),
                     "path": {1: "dense", 2: "direct"}[enc.last_path()],
                     "stage_us": {k_: round(v, 1) for k_, v in stages[name].items()}}
    enc.sync_status()
    P = sl.width * sl.height
    area = (2 * r["dx"] + 1) * (2 * r["dy"] + 1)
    dense_px_us = sum(stages["dense"][s_] for s_ in ("pool_rows", "counts", "pool_cols"))
    res["model_ns"] = {
        "pixel": 1000 * dense_px_us / P,
        "flow_dense": 1000 * stages["dense"]["gather"] / nK,
        "flow_window": 1000 * stages["direct"]["gather"] / (nK * area)}
    enc.close()
    return res


def recipes_leg(args, mode, stream):
    """The paper's four parameter recipes (window radii 8/10, delta_t 16/12 ms,
    640x480, D = 64) on the 640x480 2M-event slice, each with its pooling
    shapes autotuned for its window; flows/s per recipe."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    sl, _ = synth.workload("slice-640x480-2M")
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    flow = torch.empty((sl.n, 2), dtype=torch.float32, device="cuda")
    out = {}
    for name, r in sorted(synth.RECIPES.items()):
        T, X, Y = synth.frequencies(r["D"], 0)
        w = synth.mlp_weights(r["D"], 128, 3)
        p = vk.Params(width=r["width"], height=r["height"], D=r["D"], dx=r["dx"], dy=r["dy"],
                      dt_us=r["dt_us"], t_span_us=int(sl.t.max()) - sl.t_ref)
        enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
        tuned = enc.autotune(r["width"], r["height"], stream)
        for _ in range(args.warmup):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k = max(3, args.steps // 2)
        a.record(stream)
        for _ in range(k):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / k
        enc.sync_status()
        out[name] = {"value": sl.n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "window": f"{2 * r['dx'] + 1}x{2 * r['dy'] + 1}", "dt_us": r["dt_us"],
                     "tuned_pooling": {"rows_seg": tuned[0], "rows_warps": tuned[1],
                                       "cols_seg": tuned[2], "cols_warps": tuned[3]}}
        enc.close()
    return out


def precision_leg(args, stream):
    """The precision workload: 1280x720, 4,000,000 events over 20 ms, D = 128,
    a 256 -> 128 -> 2 head.  Per mode (FP32 or FP16 storage of the pooled
    grid, BF16 or FP16 tensor-core head, and the plain FP32 form): the step
    time, and the error per output against the FP64 oracle on a sample of
    requested events (the oracle scatters every event and pools the sampled
    ones, Algorithm 1): per flow component the largest and mean absolute
    error, the flow error relative to max(|flow|, 0.25 median |flow|), and
    the encoding's relative L2 error."""
    import torch
    import oracle
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    sl, D = synth.workload("slice-1280x720-4M")
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=sl.width, height=sl.height, D=D, dx=10, dy=10, dt_us=16_000,
                  t_span_us=int(sl.t.max()) - sl.t_ref)
    x = torch.from_numpy(sl.x).cuda()
    y = torch.from_numpy(sl.y).cuda()
    t = torch.from_numpy(sl.t.view(np.int32)).cuda()
    flow = torch.empty((sl.n, 2), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(13)
    S = args.precision_sample
    K = np.sort(rng.choice(sl.n, S, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    emb_ref, _ = oracle.encode_pooled(sl.x, sl.y, sl.t, sl.t_ref, sl.width, sl.height, D, 10, 10,
                                      16_000.0, T, X, Y, K=K)
    flow_ref = oracle.mlp(emb_ref, w.W1, w.b1, w.W2, w.b2)
    oracle_s = time.perf_counter() - t0
    nr = np.linalg.norm(flow_ref, axis=1)
    res = {"workload": f"slice-1280x720-4M ({sl.n} events, 20 ms, D={D}, 21x21, 256->128->2)",
           "error_sample": f"{S} random requested events, FP64 oracle ({oracle_s:.1f} s)",
           "modes": {}}
    Kd = torch.from_numpy(K).cuda()
    modes = (("bf16", vk.MLP_BF16), ("bf16-acc16", vk.MLP_BF16 | vk.ACC_FP16),
             ("fp16", vk.MLP_FP16), ("fp16-acc16", vk.MLP_FP16 | vk.ACC_FP16),
             ("fp32", vk.MLP_FP32))
    enc = vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=vk.MLP_BF16)
    for name, m in modes:
        enc.set_mlp_mode(m)
        enc.autotune(sl.width, sl.height, stream)
        k = max(3, args.steps // 4) if m != vk.MLP_FP32 else 3
        for _ in range(args.warmup):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            enc.predict(x, y, t, sl.t_ref, out=flow, stream=stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / k
        enc.sync_status()
        f = flow[Kd].cpu().numpy().astype(np.float64)
        d = np.abs(f - flow_ref)
        rel = np.linalg.norm(f - flow_ref, axis=1) / np.maximum(nr, 0.25 * np.median(nr))
        res["modes"][name] = {
            "ms_per_step": ms, "value": sl.n / (ms * 1e-3), "unit": UNIT,
            "flow_abs_max": [float(d[:, 0].max()), float(d[:, 1].max())],
            "flow_abs_mean": [float(d[:, 0].mean()), float(d[:, 1].mean())],
            "flow_rel_max": float(rel.max()), "flow_rel_mean": float(rel.mean()),
            "flow_rel_floor": "0.25 x median |flow|"}
    emb = enc.encode(x, y, t, sl.t_ref, K=Kd).cpu().numpy().astype(np.float64)
    e_err = np.linalg.norm(emb - emb_ref, axis=1) / np.linalg.norm(emb_ref, axis=1)
    res["emb_rel_l2_max"] = float(e_err.max())
    res["emb_rel_l2_mean"] = float(e_err.mean())
    enc.sync_status()
    enc.close()
    return res


def batch_leg(args, mode, stream):
    """Uneven slices at mixed resolutions (64 slices of 16 streams, 10k-2M
    events log-uniform, 346x260 / 640x480 / 1280x720 cycled, D=64): one
    replay of a captured CUDA-graph plan of the whole batch on a canvas,
    against one predict call per slice on per-resolution contexts.  Both
    sides are autotuned; results are compared."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    t0 = time.perf_counter()
    items = synth.stream_batch(64, 16, scale=args.batch_scale)
    gen_s = time.perf_counter() - t0
    sls = [s for _, s in items]
    D, span = 64, 20_000
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)

    def ctx(W, H):
        p = vk.Params(width=W, height=H, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=span)
        return vk.Encoder(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)

    dev = [vk.Slice(torch.from_numpy(s.x).cuda(), torch.from_numpy(s.y).cuda(),
                    torch.from_numpy(s.t.view(np.int32)).cuda(), s.t_ref, s.width, s.height)
           for s in sls]
    N = sum(s.n for s in sls)
    cw_max = 8192
    _, _, cw, ch = vk.canvas_layout([s.width for s in sls], [s.height for s in sls], 10, 10, cw_max)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    big = ctx(cw_max, ch)
    flow = torch.empty((N, 2), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    plan = big.plan(dev, out=flow)
    plan_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    batch_bytes = free0 - torch.cuda.mem_get_info()[0]

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / k

    k = max(3, args.steps // 2)
    ms_graph = timed(lambda: plan.launch(stream), k)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    ctxs = {}
    for s in sls:
        if (s.width, s.height) not in ctxs:
            c = ctx(s.width, s.height)
            c.autotune(s.width, s.height, stream)
            ctxs[(s.width, s.height)] = c
    outs = [torch.empty((s.n, 2), dtype=torch.float32, device="cuda") for s in sls]
    torch.cuda.synchronize()
    plain_bytes = free1 - torch.cuda.mem_get_info()[0]

    def plain():
        launches = 0
        for s, d, o in zip(sls, dev, outs):
            c = ctxs[(s.width, s.height)]
            c.predict(d.x, d.y, d.t, s.t_ref, out=o, stream=stream)
            launches += c.last_launch_count()
        return launches

    ms_plain = timed(plain, k)
    plain_launches = plain()
    torch.cuda.synchronize()
    cat = torch.cat(outs)
    big.sync_status()
    for c in ctxs.values():
        c.sync_status()
    agree = float(((flow - cat).abs().max() / cat.abs().max()).item())
    res = {
        "workload": "stream-batch-64x16 (64 slices, 16 streams, 10k-2M events log-uniform, "
                    "346x260/640x480/1280x720 cycled, D=64)",
        "slices": len(sls), "events": N, "canvas": f"{cw}x{ch}",
        "sensor_pixels": int(sum(s.width * s.height for s in sls)),
        "value": N / (ms_graph * 1e-3), "unit": UNIT, "ms_per_batch": ms_graph,
        "kernels_per_batch": plan.kernel_count,
        "plain": {"value": N / (ms_plain * 1e-3), "ms_per_batch": ms_plain,
                  "kernels_per_batch": int(plain_launches),
                  "form": "one veckm_predict per slice, per-resolution contexts, one stream"},
        "speedup_vs_plain": ms_plain / ms_graph, "max_rel_diff_vs_plain": agree,
        "plan_create_s": plan_s, "generate_s": gen_s,
        "device_bytes": int(batch_bytes), "device_bytes_plain": int(plain_bytes),
        "device_bytes_note": "free-memory drop: canvas context + plan + flows (batch); "
                             "per-resolution contexts + flows (plain), the slices' events excluded",
        "tuned_pooling": "per geometry (autotuner), both sides"}
    plan.close()
    del big, ctxs
    torch.cuda.empty_cache()
    return res


def serving_leg(args, mode):
    """Serving: 32 sensors (346x260 / 640x480 / 1280x720 cycled) send packets
    with Poisson arrivals at 2 kHz in aggregate, packet sizes lognormal
    (median 50k events, sigma 1, clipped to [1k, 2M]); each packet is one
    slice.  The native server admits packets by device memory and batches
    whatever is waiting.  Packets come from a pre-generated pool (the event
    values do not change the work); host buffers are pinned."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    rng = np.random.default_rng(2025)
    res = [(346, 260), (640, 480), (1280, 720)]
    n_sensors, rate_hz, dur_s = 32, 2000.0, args.serve_seconds
    pool = {}
    t0 = time.perf_counter()
    for r in range(3):
        pool[r] = []
        for j in range(12):
            n = int(np.clip(np.exp(np.log(50_000) + rng.standard_normal()), 1_000, 2_000_000))
            W, H = res[r]
            sl = synth.event_slice(W, H, n, 16_000, n_edges=8, n_blobs=2, frac_blobs=0.3,
                                   frac_noise=0.05, seed=7000 + 100 * r + j)
            pool[r].append((sl, torch.from_numpy(sl.x).pin_memory(),
                            torch.from_numpy(sl.y).pin_memory(),
                            torch.from_numpy(sl.t.view(np.int32)).pin_memory(),
                            torch.zeros((sl.n, 2), dtype=torch.float32).pin_memory()))
    gen_s = time.perf_counter() - t0
    D = 64
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    p = vk.Params(width=8192, height=2048, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=16_000)
    srv = vk.Server(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode)
    # warm-up: one packet per resolution (first launches, autotuning-free defaults)
    for r in range(3):
        sl, x, y, t, o = pool[r][0]
        srv.submit(0, x, y, t, sl.t_ref, sl.width, sl.height, o)
    srv.drain()
    srv.poll(10_000)
    warm = srv.stats()
    # the arrival process
    gaps = rng.exponential(1.0 / rate_hz, int(rate_hz * dur_s * 1.2) + 16)
    arr = np.cumsum(gaps)
    arr = arr[arr < dur_s]
    sensor = rng.integers(0, n_sensors, arr.size)
    offered = 0
    refused = 0
    start = time.perf_counter()
    for k, (ta, s) in enumerate(zip(arr, sensor)):
        while time.perf_counter() - start < ta:
            pass
        r = int(s) % 3
        sl, x, y, t, o = pool[r][k % len(pool[r])]
        offered += sl.n
        if not srv.submit(int(s), x, y, t, sl.t_ref, sl.width, sl.height, o):
            refused += 1
    submit_s = time.perf_counter() - start
    srv.drain()
    comps = srv.poll(100_000)
    st = srv.stats()
    srv.close()
    lat = np.array([c["latency_ms"] for c in comps])
    bp = np.array([c["batch_packets"] for c in comps])
    ev = st["events_completed"] - warm["events_completed"]
    wall = max(submit_s, 1e-9)
    return {
        "workload": "serve-32-sensors-2kHz (Poisson arrivals, lognormal packets median 50k "
                    "sigma 1 in [1k, 2M], 346x260/640x480/1280x720, D=64, slice = packet)",
        "seconds": dur_s, "packets": int(arr.size), "streams": int(st["streams"]),
        "offered_events_per_s": offered / dur_s,
        "served_events_per_s": ev / wall, "unit": UNIT,
        "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
        "max_ms": float(lat.max()) if lat.size else None,
        "admitted": int(st["admitted"] - warm["admitted"]), "refused": int(refused),
        "batches": int(st["batches"] - warm["batches"]),
        "mean_packets_per_batch": float(bp.mean()) if bp.size else None,
        "gpu_busy_fraction": (st["gpu_busy_s"] - warm["gpu_busy_s"]) / wall,
        "latency": "submission to completion (flows in pinned host memory), host steady clock",
        "generate_s": gen_s}


def _serving_packets(rng, n_pool=12):
    """Per resolution (346x260, 640x480, 1280x720) a pool of slices with
    lognormal sizes (median 50k events, sigma 1, clipped to [1k, 2M]), each
    16 ms of a sensor's events; pinned host copies of x, y."""
    import torch
    from paper_2504_19417_gb300 import synth
    res = [(346, 260), (640, 480), (1280, 720)]
    pool = {}
    for r in range(3):
        pool[r] = []
        for j in range(n_pool):
            n = int(np.clip(np.exp(np.log(50_000) + rng.standard_normal()), 1_000, 2_000_000))
            W, H = res[r]
            sl = synth.event_slice(W, H, n, 16_000, n_edges=8, n_blobs=2, frac_blobs=0.3,
                                   frac_noise=0.05, seed=7000 + 100 * r + j)
            pool[r].append((sl, torch.from_numpy(sl.x).pin_memory(),
                            torch.from_numpy(sl.y).pin_memory()))
    return res, pool


def serving_windows_leg(args, mode):
    """Serving with resident per-sensor windows, against the plain per-packet
    path, over a sweep of offered rates.

    32 sensors (346x260 / 640x480 / 1280x720 by sensor index mod 3) send
    packets with Poisson arrivals at the offered aggregate rate, each sensor
    choosing packets uniformly; a packet holds 16 ms of its sensor's events
    (lognormal size, median 50k, sigma 1, in [1k, 2M]) and a sensor's packets
    follow each other in time.  Every packet's flows are those of its events
    against its sensor's last 32 ms (2 delta_t, Section 2.1), ending at the
    packet's last event.
      - resident: the native server keeps each sensor's window sums on the
        device (exact fixed-point add/expire) and slides them per packet;
        packets of different sensors overlap on the device.
      - plain: one veckm_predict_host per packet, in arrival order, on the
        window's events (the sensor's recent packets, gathered on the host)
        with K = the packet's events; nothing stays resident.
    Latency is from arrival (submission) to flows in pinned host memory.  A
    rate is sustained while the served event rate stays within 5% of the
    offered one; the sweep stops at the first rate an arm does not sustain."""
    import torch
    from paper_2504_19417_gb300 import synth
    from paper_2504_19417_gb300 import veckm as vk
    rng = np.random.default_rng(2026)
    t0 = time.perf_counter()
    res, pool = _serving_packets(rng)
    gen_s = time.perf_counter() - t0
    n_sensors, win, span = 32, 32_000, 16_000
    D = 64
    T, X, Y = synth.frequencies(D, 0)
    w = synth.mlp_weights(D, 128, 3)
    rates = [float(r) for r in args.serve_rates.split(",")]
    per_point = args.serve_packets

    def schedule(rate):
        g = np.random.default_rng(int(rate))
        arr = np.cumsum(g.exponential(1.0 / rate, per_point))
        sensor = g.integers(0, n_sensors, per_point)
        pick = g.integers(0, len(pool[0]), per_point)
        return arr, sensor, pick

    class Clock:  # each sensor's own time: packets follow each other, 16 ms each
        def __init__(self):
            self.next = np.full(n_sensors, 10_000_000, np.int64)

        def take(self, s):
            off = int(self.next[s])
            self.next[s] += span
            return off

    def shifted(sl, off):
        return (sl.t.astype(np.int64) - sl.t_ref + off).astype(np.uint32)

    # ---- resident windows
    p = vk.Params(width=1280, height=720, D=D, dx=10, dy=10, dt_us=16_000, t_span_us=win)
    srv = vk.Server(p, w.W1, w.b1, w.W2, w.b2, T, X, Y, mlp_mode=mode, arena_bytes=8 << 30,
                    window_us=win, window_capacity=1 << 22)
    clk = Clock()
    free_t = []  # pinned time buffers, reused once their packet completed
    held = {}

    def t_buf(n):
        for i, b in enumerate(free_t):
            if b.numel() >= n:
                return free_t.pop(i)
        return torch.empty(max(n, 1 << 16), dtype=torch.int32).pin_memory()

    out_bufs = {r: [torch.zeros((sl.n, 2), dtype=torch.float32).pin_memory() for sl, _, _ in pool[r]]
                for r in range(3)}
    tag = [0]

    def submit(s, j):
        r = s % 3
        sl, x, y = pool[r][j]
        off = clk.take(s)
        tb = t_buf(sl.n)
        tb[: sl.n].numpy().view(np.uint32)[:] = shifted(sl, off)
        tag[0] += 1
        # the flows land in a per-pool-slice buffer (values are not checked here)
        ok = srv.submit(s, x, y, tb[: sl.n], off, sl.width, sl.height, out_bufs[r][j], tag=tag[0])
        if ok:
            held[tag[0]] = tb
        else:
            free_t.append(tb)
        return ok

    lat_now = []

    def collect(wait_ms=0):
        for c in srv.poll(4096, wait_ms):
            lat_now.append(c["latency_ms"])
            b = held.pop(c["tag"], None)
            if b is not None:
                free_t.append(b)

    # warm-up: every sensor's state, created with its first packet
    for s in range(n_sensors):
        submit(s, 0)
    srv.drain()
    collect()
    resident = []
    for rate in rates:
        arr, sensor, pick = schedule(rate)
        base = srv.stats()
        lat_now.clear()
        offered = 0
        start = time.perf_counter()
        for ta, s, j in zip(arr, sensor, pick):
            while time.perf_counter() - start < ta:
                pass
            s = int(s)
            offered += pool[s % 3][int(j)][0].n
            submit(s, int(j))
            collect()
        srv.drain()
        wall = time.perf_counter() - start
        collect()
        st = srv.stats()
        ev = st["events_completed"] - base["events_completed"]
        lat = np.array(lat_now)
        resident.append({"offered_hz": rate, "packets": per_point,
                         "offered_flows_per_s": offered / float(arr[-1]),
                         "served_flows_per_s": ev / wall,
                         "refused": int(st["refused"] - base["refused"]),
                         "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)),
                         "gpu_busy_s": st["gpu_busy_s"] - base["gpu_busy_s"]})
        if ev / wall < 0.95 * offered / float(arr[-1]):
            break
    srv.close()

    # ---- plain per-packet path
    ctxs = {r: vk.Encoder(vk.Params(width=res[r][0], height=res[r][1], D=D, dx=10, dy=10,
                                    dt_us=16_000, t_span_us=3 * span), w.W1, w.b1, w.W2, w.b2,
                          T, X, Y, mlp_mode=mode) for r in range(3)}
    for r in range(3):
        ctxs[r].autotune(res[r][0], res[r][1])
    cap = 3 * 2_000_000
    hx = torch.empty(cap, dtype=torch.int16).pin_memory()
    hy = torch.empty(cap, dtype=torch.int16).pin_memory()
    ht = torch.empty(cap, dtype=torch.int32).pin_memory()
    hk = torch.empty(2_000_000, dtype=torch.int64).pin_memory()
    hf = torch.empty((2_000_000, 2), dtype=torch.float32).pin_memory()
    clk = Clock()
    recent = {s: [] for s in range(n_sensors)}  # (pool index, offset) of the last packets

    def plain_call(s, j):
        r = s % 3
        off = clk.take(s)
        sl = pool[r][j][0]
        tk = shifted(sl, off)
        t_hi = int(tk[-1])
        parts = [(pool[r][jj][0], shifted(pool[r][jj][0], oo)) for jj, oo in recent[s][-2:]]
        xs, ys, ts = [], [], []
        for psl, pt in parts:
            m = pt >= t_hi - win
            xs.append(psl.x[m]); ys.append(psl.y[m]); ts.append(pt[m])
        n0 = int(sum(a.size for a in xs))
        xs.append(sl.x); ys.append(sl.y); ts.append(tk)
        n = n0 + sl.n
        hx[:n].numpy()[:] = np.concatenate(xs)
        hy[:n].numpy()[:] = np.concatenate(ys)
        tt = np.concatenate(ts)
        ht[:n].numpy().view(np.uint32)[:] = tt
        hk[: sl.n].numpy()[:] = np.arange(n0, n, dtype=np.int64)
        ctxs[r].predict_host(hx[:n], hy[:n], ht[:n], int(tt.min()), K=hk[: sl.n],
                             out=hf[: sl.n])
        recent[s].append((j, off))
        recent[s] = recent[s][-2:]

    for s in range(n_sensors):  # warm-up, as for the server
        plain_call(s, 0)
    plain = []
    for rate in rates:
        arr, sensor, pick = schedule(rate)
        lat = []
        offered = 0
        start = time.perf_counter()
        for ta, s, j in zip(arr, sensor, pick):
            while time.perf_counter() - start < ta:
                pass
            offered += pool[int(s) % 3][int(j)][0].n
            plain_call(int(s), int(j))
            lat.append(1000.0 * (time.perf_counter() - start - ta))
        wall = time.perf_counter() - start
        lat = np.array(lat)
        plain.append({"offered_hz": rate, "packets": per_point,
                      "offered_flows_per_s": offered / float(arr[-1]),
                      "served_flows_per_s": offered / wall,
                      "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99))})
        if offered / wall < 0.95 * offered / float(arr[-1]):
            break
    for e in ctxs.values():
        e.close()

    def sustained(pts):
        ok = [q["offered_hz"] for q in pts if q["served_flows_per_s"] >= 0.95 * q["offered_flows_per_s"]]
        return max(ok) if ok else None

    return {"workload": "serve-32-sensors (Poisson arrivals, lognormal packets median 50k sigma 1 "
                        "in [1k, 2M], 16 ms per packet, 346x260/640x480/1280x720, D=64, "
                        "32 ms window per sensor)",
            "unit": UNIT, "resident": resident, "plain": plain,
            "sustained_hz": {"resident": sustained(resident), "plain": sustained(plain)},
            "latency": "arrival to flows in pinned host memory, host steady clock",
            "generate_s": gen_s}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--mode", default="fp16",
                    choices=["bf16", "fp16", "fp32", "fp16-acc16", "bf16-acc16"])
    ap.add_argument("--lean", action="store_true", help="timed device loop only (for profilers)")
    ap.add_argument("--scale", type=float, default=1.0, help="events x scale (profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=50_000)
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-slice batch leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-recipes", action="store_true", help="skip the parameter-recipe leg")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 1280x720 D=128 precision leg")
    ap.add_argument("--precision-sample", type=int, default=5_000)
    ap.add_argument("--no-autotune", action="store_true", help="default pooling launch shapes")
    ap.add_argument("--no-sparse", action="store_true", help="skip the sparse-request leg")
    ap.add_argument("--no-small", action="store_true", help="skip the 346x260 20k-event leg")
    ap.add_argument("--no-stream", action="store_true", help="skip the sliding-window leg")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-rates", default="1000,2000,4000,6000,8000,12000,16000",
                    help="offered aggregate packet rates (Hz) of the serving sweep")
    ap.add_argument("--serve-packets", type=int, default=1500,
                    help="packets per rate of the serving sweep")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="events x scale of the batch leg")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
