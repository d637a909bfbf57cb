"""Host-side model of how the per-pixel sums share pixels between warps and
which rows the bucket sort zeroes for them (no GPU).

The sums take pixel-sorted records in ranges of 128 (one warp each).  A
pixel whose records all lie inside one range is stored once by that warp;
the first pixel of a range, and the last one unless the range is the last,
may be shared with a neighbouring range and are added into instead.  The
bucket sort zeroes the rows of the pixels at sorted positions c*128, and at
c*128 + 127 unless the next position, in the same bucket, holds the same
pixel.  The model checks on adversarial orders that every pixel added into
is zeroed first and that every pixel with records is written."""
import numpy as np
import pytest

RECS = 128


def pixsum_writes(rpix):
    """(stored, added): the pixels each range stores and adds into."""
    ns = len(rpix)
    stored, added = set(), set()
    for r0 in range(0, ns, RECS):
        r1 = min(r0 + RECS, ns)
        runs = [r0] + [r for r in range(r0 + 1, r1) if rpix[r] != rpix[r - 1]]
        for i, a in enumerate(runs):
            p = int(rpix[a])
            first, last = i == 0, i == len(runs) - 1
            if first or (last and r1 < ns):
                added.add(p)
            else:
                stored.add(p)
    return stored, added


def zeroed_by_sort(rpix, bucket_of):
    z = set()
    ns = len(rpix)
    for pos in range(ns):
        m = pos % RECS
        if m == 0:
            z.add(int(rpix[pos]))
        elif m == RECS - 1:
            same_next = (pos + 1 < ns and bucket_of(rpix[pos + 1]) == bucket_of(rpix[pos])
                         and rpix[pos + 1] == rpix[pos])
            if not same_next:
                z.add(int(rpix[pos]))
    return z


def sorted_records(counts):
    return np.repeat(np.arange(len(counts)), counts)


@pytest.mark.parametrize("case", ["uniform", "hot", "single", "edges", "short"])
def test_every_added_pixel_is_zeroed_and_every_pixel_written(case):
    rng = np.random.default_rng(7)
    P, shift = 4096, 5
    if case == "uniform":
        counts = rng.poisson(3, P)
    elif case == "hot":  # a few pixels across many ranges
        counts = rng.poisson(1, P)
        counts[[5, 6, 900, 4095]] = [1000, 129, 5000, 300]
    elif case == "single":  # one pixel, the whole slice
        counts = np.zeros(P, int)
        counts[1234] = 3 * RECS + 17
    elif case == "edges":  # runs that end exactly on range edges
        counts = np.zeros(P, int)
        counts[:64] = RECS
        counts[64:128] = 1
    else:  # fewer records than one range
        counts = np.zeros(P, int)
        counts[[3, 4, 5]] = [10, 1, 7]
    rpix = sorted_records(counts)
    stored, added = pixsum_writes(rpix)
    zeroed = zeroed_by_sort(rpix, lambda p: int(p) >> shift)
    assert added <= zeroed, sorted(added - zeroed)[:10]
    assert stored | added == set(np.flatnonzero(counts).tolist())
    assert not (stored & added)
