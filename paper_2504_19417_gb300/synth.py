"""Seeded synthetic inputs: event slices, RFF frequencies and MLP weights.

This module produces inputs only.  It holds none of the encoder's arithmetic
(no phases, no pooling, no network), so that the CUDA path and the FP64 oracle
can both be fed from it without sharing any code that computes a result.

Random numbers that the method itself draws (the frequency vectors T, X, Y of
Algorithm 1, drawn as i.i.d. normals of variance sigma^2 = 25) come from
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) followed by the Box-Muller transform.  The C library
implements the same published generator on its own side for its
``freq_seed`` path; the two are compared in the tests.

The event scenes stand in for the EVIMO2 recordings the paper evaluates on
(640x480 Samsung mono camera, Section 3.3): straight edges translating at
50-500 px/s, textured discs, and uniform noise, with integer pixel
coordinates and integer microsecond timestamps, sorted by time as a camera
emits them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 seeded with ``seed``.

    SplitMix64 is counter based: output i (0-based) is mix(seed + (i+1)*gamma)
    with gamma = 0x9E3779B97F4A7C15 and the two xor-shift-multiply rounds of
    the published definition.
    """
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller over consecutive uniform pairs.

    Pair j uses u1 = U[2j], u2 = U[2j+1]; r = sqrt(-2 ln(1-u1)); it yields
    r*cos(2 pi u2) then r*sin(2 pi u2).
    """
    npair = (count + 1) // 2
    u = uniform01(seed, 2 * npair)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(2 * npair, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def frequencies(D: int, seed: int = 0, sigma2: float = 25.0):
    """T, X, Y of Algorithm 1: D i.i.d. N(0, sigma2) each, seeds seed, seed+1, seed+2."""
    s = math.sqrt(sigma2)
    return (s * normals(seed, D), s * normals(seed + 1, D), s * normals(seed + 2, D))


@dataclass
class MLPWeights:
    W1: np.ndarray  # [hidden][2D] float32, row-major
    b1: np.ndarray  # [hidden]
    W2: np.ndarray  # [2][hidden]
    b2: np.ndarray  # [2]


def mlp_weights(D: int, hidden: int = 128, seed: int = 3) -> MLPWeights:
    """Seeded FP32 weights of the 2D -> hidden -> 2 ReLU perceptron.

    Each layer is U(-1/sqrt(fan_in), 1/sqrt(fan_in)), drawn from one SplitMix64
    stream in the order W1, b1, W2, b2.
    """
    n1, n2 = hidden * 2 * D, 2 * hidden
    u = uniform01(seed, n1 + hidden + n2 + 2) * 2.0 - 1.0
    a, b = 1.0 / math.sqrt(2 * D), 1.0 / math.sqrt(hidden)
    o = 0
    W1 = (u[o:o + n1] * a).astype(np.float32).reshape(hidden, 2 * D); o += n1
    b1 = (u[o:o + hidden] * a).astype(np.float32); o += hidden
    W2 = (u[o:o + n2] * b).astype(np.float32).reshape(2, hidden); o += n2
    b2 = (u[o:o + 2] * b).astype(np.float32)
    return MLPWeights(W1, b1, W2, b2)


@dataclass
class EventSlice:
    x: np.ndarray  # int16 [n]
    y: np.ndarray  # int16 [n]
    t: np.ndarray  # uint32 [n], microseconds, non-decreasing
    p: np.ndarray  # int8 [n], +1 / -1 (carried, unused by the encoder)
    width: int
    height: int
    t_ref: int     # slice start (microseconds)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _edges(rng, W, H, span_s, n):
    """n events from straight edges translating across the sensor."""
    xs, ys, ts, ps = [], [], [], []
    diag = math.hypot(W, H)
    anchor = rng.uniform([0, 0], [W, H])
    theta = rng.uniform(0.0, math.pi)
    tang = np.array([math.cos(theta), math.sin(theta)])
    nrm = np.array([-tang[1], tang[0]])
    speed = rng.uniform(50.0, 500.0)
    phi = rng.uniform(0.0, 2 * math.pi)
    v = speed * np.array([math.cos(phi), math.sin(phi)])
    pol = 1 if float(nrm @ v) >= 0 else -1
    got = 0
    tries = 0
    while got < n and tries < 64:
        tries += 1
        m = 2 * (n - got) + 64
        t = rng.uniform(0.0, span_s, m)
        s = rng.uniform(-diag, diag, m)
        px = anchor[0] + v[0] * t + s * tang[0]
        py = anchor[1] + v[1] * t + s * tang[1]
        xi, yi = np.rint(px), np.rint(py)
        ok = (xi >= 0) & (xi < W) & (yi >= 0) & (yi < H)
        xi, yi, t = xi[ok][: n - got], yi[ok][: n - got], t[ok][: n - got]
        xs.append(xi); ys.append(yi); ts.append(t); ps.append(np.full(xi.size, pol))
        got += xi.size
    if got < n:
        return None  # the edge barely crosses the sensor: draw another
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(ps)


def _visible_edge(rng, W, H, span_s, n):
    for _ in range(64):
        r = _edges(rng, W, H, span_s, n)
        if r is not None and r[0].size == n:
            return r
    raise RuntimeError("could not place an edge on the sensor")


def _blob(rng, W, H, span_s, n):
    """n events from a textured disc translating across the sensor."""
    R = rng.uniform(10.0, 40.0)
    c0 = rng.uniform([0, 0], [W, H])
    speed = rng.uniform(50.0, 500.0)
    phi = rng.uniform(0.0, 2 * math.pi)
    v = speed * np.array([math.cos(phi), math.sin(phi)])
    rr = R * np.sqrt(rng.uniform(0, 1, 50))
    aa = rng.uniform(0, 2 * math.pi, 50)
    dots = np.stack([rr * np.cos(aa), rr * np.sin(aa)], 1)
    xs, ys, ts, ps = [], [], [], []
    got = 0
    tries = 0
    while got < n and tries < 64:
        tries += 1
        m = 2 * (n - got) + 64
        t = rng.uniform(0.0, span_s, m)
        on_dot = rng.uniform(0, 1, m) < 0.5
        ang = rng.uniform(0, 2 * math.pi, m)
        off = np.stack([R * np.cos(ang), R * np.sin(ang)], 1)
        di = rng.integers(0, 50, m)
        off[on_dot] = dots[di[on_dot]]
        px = c0[0] + v[0] * t + off[:, 0]
        py = c0[1] + v[1] * t + off[:, 1]
        pol = np.where(off @ v >= 0, 1, -1)
        pol[on_dot] = np.where(rng.uniform(0, 1, int(on_dot.sum())) < 0.5, 1, -1)
        xi, yi = np.rint(px), np.rint(py)
        ok = (xi >= 0) & (xi < W) & (yi >= 0) & (yi < H)
        k = n - got
        xs.append(xi[ok][:k]); ys.append(yi[ok][:k]); ts.append(t[ok][:k]); ps.append(pol[ok][:k])
        got += xs[-1].size
    if got < n:
        return None
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(ps)


def event_slice(width: int, height: int, n: int, span_us: int, *, n_edges: int = 8,
                n_blobs: int = 0, frac_noise: float = 0.10, frac_blobs: float = 0.0,
                seed: int = 1000, t0_us: int = 1_000_000) -> EventSlice:
    """A time-sorted slice of n events on a width x height sensor.

    Moving-edge events take (1 - frac_noise - frac_blobs) of the slice, split
    evenly over ``n_edges`` edges; textured discs take ``frac_blobs`` and
    uniform noise ``frac_noise``.  Timestamps are integer microseconds in
    [t0_us, t0_us + span_us).
    """
    rng = np.random.default_rng(seed)
    span_s = span_us * 1e-6
    n_noise = int(round(n * frac_noise))
    n_blob_total = int(round(n * frac_blobs)) if n_blobs > 0 else 0
    n_edge_total = n - n_noise - n_blob_total
    parts = []
    if n_edges > 0 and n_edge_total > 0:
        per = np.full(n_edges, n_edge_total // n_edges)
        per[: n_edge_total - per.sum()] += 1
        for m in per:
            if m > 0:
                parts.append(_visible_edge(rng, width, height, span_s, int(m)))
    else:
        n_noise += n_edge_total
    if n_blob_total > 0:
        per = np.full(n_blobs, n_blob_total // n_blobs)
        per[: n_blob_total - per.sum()] += 1
        for m in per:
            r = None
            for _ in range(64):
                r = _blob(rng, width, height, span_s, int(m))
                if r is not None:
                    break
            if r is None:
                raise RuntimeError("could not place a blob on the sensor")
            parts.append(r)
    if n_noise > 0:
        parts.append((rng.integers(0, width, n_noise).astype(np.float64),
                      rng.integers(0, height, n_noise).astype(np.float64),
                      rng.uniform(0.0, span_s, n_noise),
                      np.where(rng.uniform(0, 1, n_noise) < 0.5, 1, -1)))
    if parts:
        x = np.concatenate([q[0] for q in parts])
        y = np.concatenate([q[1] for q in parts])
        ts = np.concatenate([q[2] for q in parts])
        p = np.concatenate([q[3] for q in parts])
    else:
        x = y = ts = p = np.zeros(0)
    tu = np.minimum(np.floor(ts * 1e6), span_us - 1).astype(np.int64) + t0_us
    order = np.argsort(tu, kind="stable")
    return EventSlice(x=x[order].astype(np.int16), y=y[order].astype(np.int16),
                      t=tu[order].astype(np.uint32), p=p[order].astype(np.int8),
                      width=width, height=height, t_ref=t0_us)


# Workloads, with the shapes of the paper's setting (640x480 sensor, D=64,
# 21x21 window, delta_t = 16 ms; Algorithm 1 and the recipe table of Section 2.3).
WORKLOADS = {
    "slice-346x260-20k": dict(width=346, height=260, n=20_000, span_us=10_000, n_edges=8,
                              frac_noise=0.10, seed=1001, D=64),
    "slice-640x480-2M": dict(width=640, height=480, n=2_000_000, span_us=50_000, n_edges=32,
                             n_blobs=8, frac_blobs=0.35, frac_noise=0.05, seed=1002, D=64),
    "slice-1280x720-4M": dict(width=1280, height=720, n=4_000_000, span_us=20_000, n_edges=32,
                              n_blobs=8, frac_blobs=0.35, frac_noise=0.05, seed=1003, D=128),
}


# The parameter recipes of the paper's recipe table (Section 2.3): the
# 640x480 sensor, D = 64, window radii 8 or 10 pixels, delta_t 16 or 12 ms
# (slices of 2 delta_t).
RECIPES = {
    "640x480_32ms_C64_k8": dict(width=640, height=480, D=64, dx=8, dy=8, dt_us=16_000),
    "640x480_32ms_C64_k10": dict(width=640, height=480, D=64, dx=10, dy=10, dt_us=16_000),
    "640x480_24ms_C64_k8": dict(width=640, height=480, D=64, dx=8, dy=8, dt_us=12_000),
    "640x480_24ms_C64_k10": dict(width=640, height=480, D=64, dx=10, dy=10, dt_us=12_000),
}


def workload(name: str, scale: float = 1.0) -> tuple[EventSlice, int]:
    """The named slice (optionally with ``scale`` times the events) and its D."""
    w = dict(WORKLOADS[name])
    D = w.pop("D")
    w["n"] = max(1, int(round(w["n"] * scale)))
    return event_slice(**w), D


def stream_batch(n_slices: int = 64, n_streams: int = 16, lo: int = 10_000, hi: int = 2_000_000,
                 seed: int = 1004, scale: float = 1.0):
    """Uneven slices at mixed resolutions (346x260, 640x480, 1280x720), log-uniform sizes."""
    rng = np.random.default_rng(seed)
    res = [(346, 260), (640, 480), (1280, 720)]
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_slices))
    out = []
    for i in range(n_slices):
        W, H = res[i % 3]
        n = max(1, int(round(sizes[i] * scale)))
        out.append((i % n_streams, event_slice(W, H, n, 20_000, n_edges=16, n_blobs=4,
                                               frac_blobs=0.3, frac_noise=0.05,
                                               seed=seed * 1000 + i)))
    return out
