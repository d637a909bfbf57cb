"""The N > 1 path of bench.py on CPU: world size 2 over gloo, no GPU.

The path shards by slice (weak scaling, no data-path collective): every rank
encodes its own independent slice; the job's time is the max over ranks and
its throughput the units of all ranks over that time.  These tests run two
real processes that rendezvous on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, ws, port):
    env = dict(os.environ)
    env.update(WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), VECKM_DIST_BACKEND="gloo",
               PYTHONPATH=ROOT + os.pathsep + env.get("PYTHONPATH", ""))
    return env


_PROBE = r"""
import json, sys
import bench
dist, rank, ws, local = bench._dist()
t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)   # rank 1 is the slower one
w = bench.rank_slice_def("slice-346x260-20k", rank)
print(json.dumps({"rank": rank, "ws": ws, "max_ms": t, "seed": w["seed"], "n": w["n"],
                  "rate": bench.job_rate(ws, w["n"], 3, t)}))
dist.barrier()
dist.destroy_process_group()
"""


def _run_ranks(args, ws=2, timeout=240):
    port = _free_port()
    procs = [subprocess.Popen(args, cwd=ROOT, env=_env(r, ws, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(ws)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        outs.append((p.returncode, o, e))
    return outs


def test_max_over_ranks_seeds_and_job_rate_world_size_2():
    outs = _run_ranks([sys.executable, "-c", _PROBE])
    res = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        res.append(json.loads(o.strip().splitlines()[-1]))
    res.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1] and all(d["ws"] == 2 for d in res)
    # every rank sees the slowest rank's time
    assert all(d["max_ms"] == 15.0 for d in res)
    # independent slices: same shape, different seeds
    assert res[0]["seed"] != res[1]["seed"] and res[0]["n"] == res[1]["n"]
    # whole-job rate: both ranks' units over the max time
    assert res[0]["rate"] == pytest.approx(2 * res[0]["n"] * 3 / 0.015)


def test_reference_arm_prints_once_under_two_ranks():
    args = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
            "--warmup", "0", "--workload", "slice-346x260-20k", "--ref-sample", "300"]
    outs = _run_ranks(args)
    rc0, o0, e0 = outs[0]
    rc1, o1, e1 = outs[1]
    assert rc0 == 0, e0[-2000:]
    assert rc1 == 0, e1[-2000:]
    lines0 = [l for l in o0.splitlines() if l.startswith("{")]
    lines1 = [l for l in o1.splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and lines1 == []
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_job_rate_is_weak_scaling_arithmetic():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.job_rate(1, 1000, 10, 1000.0) == pytest.approx(10_000)
    assert bench.job_rate(4, 1000, 10, 1000.0) == pytest.approx(40_000)
    assert bench.max_over_ranks(None, 3.5) == 3.5
    a = bench.rank_slice_def("slice-640x480-2M", 0, 0.5)
    b = bench.rank_slice_def("slice-640x480-2M", 3, 0.5)
    assert a["n"] == b["n"] == 1_000_000 and b["seed"] - a["seed"] == 300
