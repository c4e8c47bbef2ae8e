"""The link stage's slope window contains every pair that passes C1.

The CUDA link kernel tests a pair of cells a = (h0, h1), b = (h1, h2) with the exact
cuts only when their r-z slopes satisfy
    |t_a - t_b| <= min((rz0 + rz1 cotmax)/d1 + (rz0 + rz1 |t_a|)/m,
                       (rz0 + rz1 |t_a|)(1/d1 + 1/m) / (1 - rz1/d1)) * 1.01 + 1e-3
(d1 = r1 - r0, m <= r2 - r1, the second term only where d1 > rz1), with slopes from
approximate float32 quotients (a few ulp).  This file checks that inequality against C1
evaluated in float32 exactly as the oracle does, on random and on boundary-hugging
triplets, with D4 (|t_b| <= cotmax) applied as in the chain, after moving both slopes
apart by 4 ulp relative each.
"""

import numpy as np

f32 = np.float32


def c1_pass(z0, r0, z1, r1, z2, r2, rz0, rz1):
    """C1 in float32, the oracle's operation order (no contraction)."""
    lhs = np.abs((z1 - z0) * (r2 - r0) - (z2 - z0) * (r1 - r0))
    rhs = rz0 * (r2 - r0) + rz1 * np.abs(z2 - z0)
    return lhs <= rhs


def window(ta, d1, m, rz0, rz1, cotmax):
    ta, d1, m = (np.asarray(v, np.float64) for v in (ta, d1, m))
    ua = rz0 + rz1 * np.abs(ta)
    w_old = (rz0 + rz1 * cotmax) / d1 + ua / m
    shrink = 1.0 - rz1 / d1
    w_new = np.where(shrink > 0, ua * (1.0 / d1 + 1.0 / m) / np.where(shrink > 0, shrink, 1.0),
                     np.inf)
    return np.minimum(w_old, w_new) * 1.01 + 1e-3


def _check(cuts, r0, r1, r2, z0, z1, z2):
    rz0, rz1, cotmax = f32(cuts["rz0"]), f32(cuts["rz1"]), f32(cuts["cotmax"])
    ok = c1_pass(z0, r0, z1, r1, z2, r2, rz0, rz1)
    ta = ((z1 - z0) / (r1 - r0)).astype(np.float64)   # float32 slopes
    tb = ((z2 - z1) / (r2 - r1)).astype(np.float64)
    d4 = np.abs(z2 - z1) <= cotmax * (r2 - r1)
    sel = ok & d4
    w = window(ta, r1 - r0, r2 - r1, float(rz0), float(rz1), float(cotmax))
    ulp4 = 4 * 2.0 ** -23
    d = np.abs(ta - tb) + ulp4 * (np.abs(ta) + np.abs(tb))  # approximate quotients
    assert sel.sum() > 1000
    assert np.all(d[sel] <= w[sel]), (d[sel] - w[sel]).max()


def test_window_contains_c1_random(cuts):
    rng = np.random.default_rng(11)
    n = 400_000
    r0 = rng.uniform(2.0, 12.0, n).astype(f32)
    r1 = (r0 + rng.uniform(0.02, 12.0, n)).astype(f32)
    r2 = (r1 + rng.uniform(0.02, 12.0, n)).astype(f32)
    ta = rng.uniform(-7, 7, n)
    z0 = rng.uniform(-25, 25, n).astype(f32)
    z1 = (z0 + ta * (r1 - r0)).astype(f32)
    tb = ta + rng.normal(0, 0.05, n) * rng.choice([1, 10], n)
    z2 = (z1 + tb * (r2 - r1)).astype(f32)
    _check(cuts, r0, r1, r2, z0, z1, z2)


def test_window_contains_c1_at_the_boundary(cuts):
    """t_b placed where C1 holds with equality (in float64), then nudged inwards."""
    rng = np.random.default_rng(12)
    n = 400_000
    rz0, rz1 = float(cuts["rz0"]), float(cuts["rz1"])
    r0 = rng.uniform(2.0, 12.0, n)
    d1 = rng.choice([0.015, 0.05, 0.5, 3.0, 10.0], n) * rng.uniform(0.9, 1.1, n)
    d2 = rng.choice([0.015, 0.05, 0.5, 3.0, 10.0], n) * rng.uniform(0.9, 1.1, n)
    ta = rng.uniform(-6.5, 6.5, n)
    s = rng.choice([-1.0, 1.0], n)
    # d1 d2 |ta - tb| = rz0 (d1 + d2) + rz1 |ta d1 + tb d2|, solved for tb = ta + s*delta
    delta = np.zeros(n)
    for sign in (1.0, -1.0):   # the sign of ta d1 + tb d2 at the solution
        den = d1 * d2 - sign * s * rz1 * d2
        cand = (rz0 * (d1 + d2) + sign * rz1 * ta * (d1 + d2)) / den
        good = (cand > 0) & (den > 0) & (np.sign(ta * (d1 + d2) + s * cand * d2) == sign)
        delta = np.where(good & (delta == 0), cand, delta)
    delta *= 1 - 1e-6
    tb = ta + s * delta
    z0 = rng.uniform(-20, 20, n)
    r1 = r0 + d1
    r2 = r1 + d2
    z1 = z0 + ta * d1
    z2 = z1 + tb * d2
    _check(cuts, *(v.astype(f32) for v in (r0, r1, r2, z0, z1, z2)))


def _bucket(x, tmin, scale, nb=128):
    """The link kernel's slope bucket: trunc((x - tmin) * scale) in float32, clamped."""
    v = (x.astype(f32) - f32(tmin)).astype(f32) * f32(scale)
    return np.clip(np.trunc(v.astype(f32)), 0, nb - 1).astype(np.int64)


def test_bucket_range_contains_window():
    """Outgoing slopes are counting-sorted into 128 buckets spanning their range, and an
    incoming cell visits the buckets of t_a - w2 .. t_a + w2 with w2 = 1.001 w + 1e-5:
    every staged slope with |t_a - t_b| <= w (float32) lies in a visited bucket, for
    windows down to 1e-3 and slopes up to the largest |t| the cuts allow."""
    rng = np.random.default_rng(13)
    for trial in range(400):
        spread = rng.choice([1e-4, 0.01, 0.5, 5.0, 13.0])
        t0 = rng.uniform(-7, 7 - spread)
        tb = (t0 + rng.uniform(0, spread, rng.integers(1, 129))).astype(f32)
        tmin, tmax = tb.min(), tb.max()
        scale = f32(128) / f32(tmax - tmin) if tmax - tmin > 1e-6 else f32(0)
        kb = _bucket(tb, tmin, scale)
        ta = (rng.uniform(t0 - 0.1, t0 + spread + 0.1, 200)).astype(f32)
        w = f32(1e-3) + rng.choice([0.0, 1e-3, 0.05, 0.3], 200).astype(f32)
        w2 = (w * f32(1.001) + f32(1e-5)).astype(f32)
        lo = _bucket((ta - w2).astype(f32), tmin, scale)
        hi = _bucket((ta + w2).astype(f32), tmin, scale)
        inside = np.abs((tb[None, :] - ta[:, None]).astype(f32)) <= w[:, None]
        ok = (kb[None, :] >= lo[:, None]) & (kb[None, :] <= hi[:, None])
        assert np.all(ok[inside]), trial
