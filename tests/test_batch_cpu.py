"""Batches without a GPU: the canvas layout of the library (host logic) and
the reading behind batching, checked on the FP64 oracle.

Batching rests on two properties of the encoding (Eq. emb, Eq. 16-17):
coordinates and times enter only as differences inside a window, so a sensor
moved to an offset of a larger canvas, with its own time origin, encodes as
on its own; and a gap of at least dx columns / dy rows keeps every window
inside its own sensor.  The last tests check exactly that with the oracle, on
offsets produced by the library's layout."""
import numpy as np
import pytest

import oracle
from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk


def _rects_apart(ox, oy, w, h, gx, gy):
    for i in range(len(w)):
        for j in range(i + 1, len(w)):
            apart_x = ox[i] + w[i] + gx <= ox[j] or ox[j] + w[j] + gx <= ox[i]
            apart_y = oy[i] + h[i] + gy <= oy[j] or oy[j] + h[j] + gy <= oy[i]
            if not (apart_x or apart_y):
                return False
    return True


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_layout_places_sensors_apart_inside_the_canvas(seed):
    rng = np.random.default_rng(seed)
    n = 40
    w = rng.integers(1, 1300, n).astype(np.int32)
    h = rng.integers(1, 800, n).astype(np.int32)
    gx, gy, maxw = 10, 7, 4096
    ox, oy, cw, ch = vk.canvas_layout(w, h, gx, gy, maxw)
    assert cw <= maxw
    assert np.all(ox >= 0) and np.all(oy >= 0)
    assert np.all(ox + w <= cw) and np.all(oy + h <= ch)
    assert cw == int(np.max(ox + w)) and ch == int(np.max(oy + h))
    assert _rects_apart(ox, oy, w, h, gx, gy)
    again = vk.canvas_layout(w, h, gx, gy, maxw)
    assert np.array_equal(again[0], ox) and np.array_equal(again[1], oy)


def test_layout_shelves_follow_height_order():
    w = np.array([100, 100, 100], np.int32)
    h = np.array([10, 30, 20], np.int32)
    ox, oy, cw, ch = vk.canvas_layout(w, h, 5, 5, 1000)
    # one shelf, tallest first: sensor 1 at x=0, sensor 2 next, then sensor 0
    assert list(ox) == [210, 0, 105] and list(oy) == [0, 0, 0]
    assert (cw, ch) == (310, 30)
    ox, oy, cw, ch = vk.canvas_layout(w, h, 5, 5, 250)
    assert list(oy) == [35, 0, 0] and list(ox) == [0, 0, 105]
    assert (cw, ch) == (205, 45)


def test_layout_edge_cases():
    ox, oy, cw, ch = vk.canvas_layout([], [], 10, 10, 100)
    assert (cw, ch) == (0, 0) and ox.size == 0
    with pytest.raises(vk.VeckmError) as ei:
        vk.canvas_layout([101], [5], 10, 10, 100)
    assert ei.value.status == vk.VECKM_EINVAL
    with pytest.raises(vk.VeckmError):
        vk.canvas_layout([0], [5], 10, 10, 100)
    ox, oy, cw, ch = vk.canvas_layout([100], [5], 10, 10, 100)
    assert (cw, ch) == (100, 5)


@pytest.mark.parametrize("w,h,maxw", [(346, 260, 640), (640, 480, 640), (1, 1, 5), (97, 61, 4096)])
def test_one_slice_is_its_own_canvas(w, h, maxw):
    # a batch or plan of one slice runs the pipeline on the slice's own
    # buffers: that needs the slice at the origin of a canvas of its size
    ox, oy, cw, ch = vk.canvas_layout([w], [h], 10, 10, maxw)
    assert (int(ox[0]), int(oy[0]), cw, ch) == (0, 0, w, h)


def _slices(seed):
    rng = np.random.default_rng(seed)
    out = []
    for i, (W, H) in enumerate([(37, 29), (52, 20), (23, 41), (30, 30)]):
        n = int(rng.integers(150, 400))
        sl = synth.event_slice(W, H, n, 9_000, n_edges=3, frac_noise=0.2,
                               seed=seed * 10 + i, t0_us=1_000_000 + 777_777 * i)
        out.append(sl)
    return out


@pytest.mark.parametrize("dx,dy", [(4, 3), (5, 5), (0, 2)])
def test_oracle_on_the_canvas_equals_each_slice_alone(dx, dy):
    D = 16
    T, X, Y = synth.frequencies(D, 0)
    sls = _slices(dx * 7 + dy)
    ox, oy, cw, ch = vk.canvas_layout([s.width for s in sls], [s.height for s in sls], dx, dy, 90)
    xs, ys, ts = [], [], []
    for s, a, b in zip(sls, ox, oy):
        xs.append(s.x.astype(np.int64) + a)
        ys.append(s.y.astype(np.int64) + b)
        ts.append(s.t.astype(np.int64) - s.t_ref)  # each slice keeps its own time origin
    cx = np.concatenate(xs).astype(np.int16)
    cy = np.concatenate(ys).astype(np.int16)
    ct = np.concatenate(ts).astype(np.uint32)
    emb_c, cnt_c = oracle.encode_pooled(cx, cy, ct, 0, cw, ch, D, dx, dy, 8_000.0, T, X, Y)
    start = 0
    for s in sls:
        emb_s, cnt_s = oracle.encode_pooled(s.x, s.y, s.t, s.t_ref, s.width, s.height, D, dx, dy,
                                            8_000.0, T, X, Y)
        rows = slice(start, start + s.n)
        assert np.array_equal(cnt_c[rows], cnt_s)
        assert np.max(np.abs(emb_c[rows] - emb_s)) < 1e-12
        start += s.n


def test_a_gap_narrower_than_the_window_would_mix_slices():
    # the converse: with one column less than dx between two sensors, some
    # windows reach the neighbour and the canvas encoding changes
    D, dx, dy = 16, 4, 3
    T, X, Y = synth.frequencies(D, 0)
    a = synth.event_slice(20, 20, 300, 9_000, n_edges=2, frac_noise=1.0, seed=5)
    b = synth.event_slice(20, 20, 300, 9_000, n_edges=2, frac_noise=1.0, seed=6)
    off = 20 + dx - 1
    cx = np.concatenate([a.x, b.x.astype(np.int64) + off]).astype(np.int16)
    cy = np.concatenate([a.y, b.y]).astype(np.int16)
    ct = np.concatenate([a.t - a.t_ref, b.t - b.t_ref]).astype(np.uint32)
    emb_c, _ = oracle.encode_pooled(cx, cy, ct, 0, off + 20, 20, D, dx, dy, 8_000.0, T, X, Y)
    emb_a, _ = oracle.encode_pooled(a.x, a.y, a.t, a.t_ref, 20, 20, D, dx, dy, 8_000.0, T, X, Y)
    assert np.max(np.abs(emb_c[:a.n] - emb_a)) > 1e-3
