"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test fixes a property that the paper or plain mathematics determines:
  * the adjacency form (Eq. emb) and Algorithm 1's pooled form agree
    (the derivation of Eq. 13-17 says they are equal in exact arithmetic);
  * closed forms of Eq. (emb): an isolated event encodes to all ones, a pair
    at offset delta to (1 + exp(i w.delta))/2, m events at one pixel to the
    mean of their temporal phases, coincident events to all ones;
  * invariance under integer translation of x, y, t and the X -> -X map
    under reflection (Eq. emb depends on differences only);
  * window counts equal a brute-force count (Eq. 1 and Eq. 17);
  * Lemma 1: (1/D)<emb, phi(q)> approaches a Gaussian kernel density as D grows;
  * the perceptron on a hand-worked example and its zero-weight closed form;
  * SplitMix64's published outputs and the N(0, 25) frequency law (Alg. 1
    frequencies).
A planted mistake in any one of the oracle's steps (a dropped term, a sign,
a swapped axis, a wrong normaliser) breaks at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _freqs(D, seed=0):
    return synth.frequencies(D, seed)


def _random_events(rng, W, H, n, span, dup_frac=0.1):
    x = rng.integers(0, W, n)
    y = rng.integers(0, H, n)
    t = rng.integers(0, span, n)
    # force duplicates (same pixel, some same time) and border events
    m = int(n * dup_frac)
    if m:
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        x[dst], y[dst] = x[src], y[src]
        t[dst[: m // 2]] = t[src[: m // 2]]
    x[:4] = [0, W - 1, 0, W - 1]
    y[:4] = [0, 0, H - 1, H - 1]
    o = np.argsort(t, kind="stable")
    return x[o].astype(np.int16), y[o].astype(np.int16), (t[o] + 5000).astype(np.uint32)


@pytest.mark.parametrize("W,H,n,D,dx,dy", [(48, 40, 1500, 16, 10, 10), (33, 29, 800, 8, 3, 7),
                                           (64, 64, 2000, 12, 8, 8), (20, 12, 300, 4, 0, 2)])
def test_adjacency_form_equals_pooled_form(W, H, n, D, dx, dy):
    rng = np.random.default_rng(W * 1000 + n)
    x, y, t = _random_events(rng, W, H, n, 30_000)
    T, X, Y = _freqs(D, 7)
    args = (x, y, t, 5000, W, H, D, dx, dy, 16_000.0, T, X, Y)
    e1, c1 = oracle.encode_direct(*args)
    e2, c2 = oracle.encode_pooled(*args)
    assert np.array_equal(c1, c2)
    assert np.max(np.abs(e1 - e2)) < 1e-12


def test_counts_equal_brute_force():
    rng = np.random.default_rng(5)
    W, H, n, dx, dy = 30, 25, 400, 4, 6
    x, y, t = _random_events(rng, W, H, n, 1000)
    T, X, Y = _freqs(4)
    _, c = oracle.encode_pooled(x, y, t, 5000, W, H, 4, dx, dy, 16_000.0, T, X, Y)
    xi, yi = x.astype(int), y.astype(int)
    for k in range(n):
        ref = sum(1 for j in range(n) if abs(xi[j] - xi[k]) <= dx and abs(yi[j] - yi[k]) <= dy)
        assert c[k] == ref


@pytest.mark.parametrize("form", ["direct", "pooled"])
def test_isolated_event_encodes_to_all_ones(form):
    fn = oracle.encode_direct if form == "direct" else oracle.encode_pooled
    D = 32
    T, X, Y = _freqs(D)
    # events more than a window apart: each sees only itself
    x = np.array([2, 30, 58, 2], np.int16)
    y = np.array([3, 30, 3, 50], np.int16)
    t = np.array([7000, 9000, 12345, 40000], np.uint32)
    e, c = fn(x, y, t, 0, 64, 64, D, 10, 10, 16_000.0, T, X, Y)
    assert np.all(c == 1)
    assert np.max(np.abs(e[:, :D] - 1.0)) < 1e-15
    assert np.max(np.abs(e[:, D:])) < 1e-15


@pytest.mark.parametrize("form", ["direct", "pooled"])
@pytest.mark.parametrize("off", [(1234, 3, -2), (-500, -10, 10), (0, 1, 0), (20000, 0, -7)])
def test_pair_closed_form(form, off):
    fn = oracle.encode_direct if form == "direct" else oracle.encode_pooled
    D, dx, dy, dt = 24, 10, 10, 16_000.0
    T, X, Y = _freqs(D, 11)
    a = (30_000, 20, 20)
    b = (a[0] + off[0], a[1] + off[1], a[2] + off[2])
    x = np.array([a[1], b[1]], np.int16)
    y = np.array([a[2], b[2]], np.int16)
    t = np.array([a[0], b[0]], np.uint32)
    e, c = fn(x, y, t, 0, 48, 48, D, dx, dy, dt, T, X, Y)
    assert list(c) == [2, 2]
    ang = off[0] / dt * T + off[1] / dx * X + off[2] / dy * Y
    want_a = (1.0 + np.exp(1j * ang)) / 2.0
    want_b = (1.0 + np.exp(-1j * ang)) / 2.0
    got_a = e[0, :D] + 1j * e[0, D:]
    got_b = e[1, :D] + 1j * e[1, D:]
    assert np.max(np.abs(got_a - want_a)) < 1e-13
    assert np.max(np.abs(got_b - want_b)) < 1e-13


@pytest.mark.parametrize("form", ["direct", "pooled"])
def test_same_pixel_events_mean_temporal_phase(form):
    fn = oracle.encode_direct if form == "direct" else oracle.encode_pooled
    D, dt = 16, 16_000.0
    T, X, Y = _freqs(D, 3)
    ts = np.array([1000, 1500, 4000, 9000, 31000], np.uint32)
    m = ts.size
    x = np.full(m, 9, np.int16)
    y = np.full(m, 4, np.int16)
    e, c = fn(x, y, ts, 1000, 20, 10, D, 10, 10, dt, T, X, Y)
    assert np.all(c == m)
    for k in range(m):
        want = np.mean(np.exp(1j * np.outer((ts.astype(float) - ts[k]) / dt, T)), axis=0)
        assert np.max(np.abs(e[k, :D] + 1j * e[k, D:] - want)) < 1e-14


def test_coincident_events_encode_to_all_ones():
    D = 8
    T, X, Y = _freqs(D)
    n = 6
    x = np.full(n, 5, np.int16)
    y = np.full(n, 6, np.int16)
    t = np.full(n, 777, np.uint32)
    for fn in (oracle.encode_direct, oracle.encode_pooled):
        e, c = fn(x, y, t, 0, 10, 10, D, 2, 2, 16_000.0, T, X, Y)
        assert np.all(c == n)
        assert np.max(np.abs(e[:, :D] - 1)) < 1e-14 and np.max(np.abs(e[:, D:])) < 1e-14


@pytest.mark.parametrize("form", ["direct", "pooled"])
def test_integer_translation_invariance(form):
    fn = oracle.encode_direct if form == "direct" else oracle.encode_pooled
    rng = np.random.default_rng(9)
    W, H, D = 40, 30, 16
    x = rng.integers(0, 25, 500)
    y = rng.integers(0, 20, 500)
    t = np.sort(rng.integers(0, 20000, 500))
    T, X, Y = _freqs(D, 2)
    base = fn(x.astype(np.int16), y.astype(np.int16), t.astype(np.uint32), 0, W, H, D, 6, 4,
              12_000.0, T, X, Y)
    for sx, sy, st in [(15, 10, 777), (3, 0, 123456), (0, 9, 1)]:
        sh = fn((x + sx).astype(np.int16), (y + sy).astype(np.int16), (t + st).astype(np.uint32),
                st, W, H, D, 6, 4, 12_000.0, T, X, Y)
        assert np.array_equal(base[1], sh[1])
        assert np.max(np.abs(base[0] - sh[0])) < 1e-12


def test_reflection_maps_X_to_minus_X():
    rng = np.random.default_rng(4)
    W, H, D = 32, 24, 12
    x = rng.integers(0, W, 300)
    y = rng.integers(0, H, 300)
    t = np.sort(rng.integers(0, 9000, 300))
    T, X, Y = _freqs(D, 5)
    a, _ = oracle.encode_pooled(x.astype(np.int16), y.astype(np.int16), t.astype(np.uint32), 0,
                                W, H, D, 5, 5, 10_000.0, T, X, Y)
    b, _ = oracle.encode_pooled((W - 1 - x).astype(np.int16), y.astype(np.int16),
                                t.astype(np.uint32), 0, W, H, D, 5, 5, 10_000.0, T, -X, Y)
    assert np.max(np.abs(a - b)) < 1e-12


def test_swapping_axes_swaps_frequencies():
    # x<->y with X<->Y and dx<->dy leaves Eq. (emb) unchanged: catches a swapped axis
    rng = np.random.default_rng(8)
    W, H, D = 30, 22, 10
    x = rng.integers(0, W, 250)
    y = rng.integers(0, H, 250)
    t = np.sort(rng.integers(0, 9000, 250))
    T, X, Y = _freqs(D, 6)
    a, ca = oracle.encode_pooled(x.astype(np.int16), y.astype(np.int16), t.astype(np.uint32), 0,
                                 W, H, D, 3, 6, 10_000.0, T, X, Y)
    b, cb = oracle.encode_pooled(y.astype(np.int16), x.astype(np.int16), t.astype(np.uint32), 0,
                                 H, W, D, 6, 3, 10_000.0, T, Y, X)
    assert np.array_equal(ca, cb)
    assert np.max(np.abs(a - b)) < 1e-12


def test_subset_K_equals_rows_of_full():
    rng = np.random.default_rng(12)
    W, H, D = 40, 40, 8
    x, y, t = _random_events(rng, W, H, 600, 20000)
    T, X, Y = _freqs(D)
    full, cf = oracle.encode_pooled(x, y, t, 5000, W, H, D, 10, 10, 16_000.0, T, X, Y)
    K = np.array([599, 0, 17, 17, 300], np.int64)
    sub, cs = oracle.encode_pooled(x, y, t, 5000, W, H, D, 10, 10, 16_000.0, T, X, Y, K=K)
    assert np.array_equal(sub, full[K]) and np.array_equal(cs, cf[K])
    sub2, _ = oracle.encode_direct(x, y, t, 5000, W, H, D, 10, 10, 16_000.0, T, X, Y, K=K)
    assert np.max(np.abs(sub2 - full[K])) < 1e-12


def test_kde_limit_lemma1():
    """Lemma 1: (1/D) Re<emb_0, phi(q)> -> (1/n) sum_k exp(-sigma^2 |u_k - q|^2 / 2).

    With frequencies of variance sigma^2 the kernel is the normal
    characteristic function, i.e. bandwidth 1/sigma in normalised units.
    """
    D, sigma2 = 8192, 25.0
    T, X, Y = synth.frequencies(D, 20, sigma2)
    rng = np.random.default_rng(1)
    n = 40
    x = (16 + rng.integers(-3, 4, n)).astype(np.int16)
    y = (16 + rng.integers(-3, 4, n)).astype(np.int16)
    t = np.sort(rng.integers(0, 4000, n)).astype(np.uint32)
    dx = dy = 10
    dt = 16_000.0
    e, _ = oracle.encode_pooled(x, y, t, 0, 32, 32, D, dx, dy, dt, T, X, Y, K=np.array([0]))
    u = np.stack([(t.astype(float) - t[0]) / dt, (x.astype(float) - x[0]) / dx,
                  (y.astype(float) - y[0]) / dy], 1)
    worst = 0.0
    for q in [u[0], u[5], u[17], u[5] + 0.03, np.array([0.05, 0.1, -0.1])]:
        g = np.mean(np.exp(-sigma2 * np.sum((u - q) ** 2, 1) / 2.0))
        got = oracle.kde_query(e[0], T, X, Y, *q)
        worst = max(worst, abs(got - g))
    assert worst < 5.0 / math.sqrt(D)


def test_mlp_hand_worked():
    g = json.load(open(os.path.join(GOLD, "mlp_tiny.json")))
    W1, b1 = np.array(g["W1"], np.float32), np.array(g["b1"], np.float32)
    W2, b2 = np.array(g["W2"], np.float32), np.array(g["b2"], np.float32)
    emb = np.array([c["emb"] for c in g["cases"]])
    flow = oracle.mlp(emb, W1, b1, W2, b2)
    assert np.array_equal(flow, np.array([c["flow"] for c in g["cases"]]))


def test_mlp_zero_first_layer_closed_form():
    D, Hd = 8, 128
    w = synth.mlp_weights(D, Hd, 3)
    emb = np.random.default_rng(0).uniform(-1, 1, (10, 2 * D))
    flow = oracle.mlp(emb, np.zeros_like(w.W1), w.b1, w.W2, w.b2)
    want = w.W2.astype(np.float64) @ np.maximum(w.b1.astype(np.float64), 0) + w.b2
    assert np.max(np.abs(flow - want[None, :])) < 1e-12


def test_mlp_reduces_to_matmul():
    D, Hd = 16, 128
    w = synth.mlp_weights(D, Hd, 3)
    emb = np.random.default_rng(1).uniform(-1, 1, (50, 2 * D))
    flow = oracle.mlp(emb, w.W1, w.b1, w.W2, w.b2)
    h = np.maximum(emb @ w.W1.astype(np.float64).T + w.b1, 0.0)
    want = h @ w.W2.astype(np.float64).T + w.b2
    assert np.max(np.abs(flow - want)) < 1e-12


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    for case in g["cases"]:
        want = [int(v, 0) for v in case["outputs"]]
        got = [int(v) for v in synth.splitmix64(case["seed"], len(want))]
        assert got == want


def test_frequency_law():
    z = synth.normals(0, 200_000)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    # Kolmogorov-Smirnov distance to the standard normal CDF
    zs = np.sort(z)
    cdf = 0.5 * (1 + np.vectorize(math.erf)(zs / math.sqrt(2)))
    ks = np.max(np.abs(cdf - np.arange(1, zs.size + 1) / zs.size))
    assert ks < 1.63 / math.sqrt(zs.size)  # 1% level
    T, X, Y = synth.frequencies(4096, 0, 25.0)
    for v in (T, X, Y):
        assert abs(v.var() - 25.0) < 5 * 25.0 * math.sqrt(2.0 / v.size)
    assert not np.allclose(T, X) and not np.allclose(X, Y)


def test_out_of_range_events_are_rejected():
    T, X, Y = _freqs(4)
    with pytest.raises(oracle.OracleError):
        oracle.encode_pooled(np.array([10], np.int16), np.array([0], np.int16),
                             np.array([5], np.uint32), 0, 10, 10, 4, 2, 2, 100.0, T, X, Y)
    with pytest.raises(oracle.OracleError):
        oracle.encode_direct(np.array([1], np.int16), np.array([1], np.int16),
                             np.array([5], np.uint32), 6, 10, 10, 4, 2, 2, 100.0, T, X, Y)
