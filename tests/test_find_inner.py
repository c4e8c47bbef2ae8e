"""The link-target pass finds a link's target cell as the position of an inner hit in a
segment of cells ordered by inner hit (`find_inner` in the link kernel's source): a guess
from the segment's first and last inner hits, the eight cells around it read at once,
and a bisection of the side beyond them when the guess missed.  This file restates that
search over plain integers and checks it against numpy's lower bound on segments of
every size up to 80 and on the shapes the doublet search gives (inner hits spread over
one window, or over two windows when an azimuthal window wraps around the layer's first
bin, with a large gap between them), for hits that are in the segment, between its
entries, and outside it.
"""

import numpy as np


def find_inner(cells, lo, hi, h):
    """The kernel's search: (position, found)."""
    end = hi
    w0 = lo
    if hi - lo > 8:
        f, la = int(cells[lo]), int(cells[hi - 1])
        if h <= f:
            return lo, h == f
        if h > la:
            return hi, False
        g = lo + (h - f) * (hi - 1 - lo) // (la - f)
        w0 = min(max(g, lo + 3) - 3, hi - 8)
    less, eq = 0, False
    for k in range(8):
        v = int(cells[w0 + k]) if w0 + k < hi else 0xFFFFFFFF
        less += v < h
        eq |= v == h
    if hi - lo <= 8 or 0 < less < 8:
        return w0 + less, eq
    if less == 0:
        hi = w0
    else:
        lo = w0 + 8
    while lo < hi:
        mid = (lo + hi) >> 1
        if cells[mid] < h:
            lo = mid + 1
        else:
            hi = mid
    return lo, lo < end and cells[lo] == h


def _segments(rng):
    for n in range(0, 81):
        yield np.sort(rng.choice(10_000, n, replace=False))
    for _ in range(300):
        n = int(rng.integers(9, 400))
        kind = rng.integers(3)
        if kind == 0:   # one window, even spread
            base = int(rng.integers(0, 1 << 20))
            seg = base + np.sort(rng.choice(4 * n, n, replace=False))
        elif kind == 1:  # two windows around the wrap of the azimuth, far apart
            a = int(rng.integers(1, n))
            seg = np.concatenate([np.sort(rng.choice(500, a, replace=False)),
                                  40_000 + np.sort(rng.choice(500, n - a, replace=False))])
        else:            # clustered: dense runs separated by gaps
            runs = [int(rng.integers(0, 1 << 16)) + np.arange(int(rng.integers(1, 20)))
                    for _ in range(int(rng.integers(2, 12)))]
            seg = np.unique(np.concatenate(runs))
        yield np.asarray(seg, np.int64)


def test_find_inner_equals_lower_bound():
    rng = np.random.default_rng(31)
    checked = 0
    for seg in _segments(rng):
        pad = int(rng.integers(0, 5))
        cells = np.concatenate([np.full(pad, -1), seg, np.full(3, 1 << 40)])
        lo, hi = pad, pad + seg.size
        queries = set(seg.tolist())
        if seg.size:
            queries |= {int(seg[0]) - 1, int(seg[-1]) + 1, 0}
            queries |= set((seg[:-1] + 1).tolist()) if seg.size > 1 else set()
        queries |= set(rng.integers(0, (int(seg[-1]) + 10) if seg.size else 100, 20).tolist())
        for h in queries:
            if h < 0:
                continue
            want = lo + int(np.searchsorted(seg, h, side="left"))
            got, found = find_inner(cells, lo, hi, int(h))
            assert got == want, (seg.size, h)
            assert found == (want < hi and cells[want] == h)
            checked += 1
    assert checked > 20_000
