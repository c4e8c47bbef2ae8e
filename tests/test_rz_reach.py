"""The doublet searches skip a layer for a hit when no point of the layer's r-z extent can
pass D2 and D3 with the hit (`rz_box_reachable` in the kernels' shared header).  This
file restates that test in float32 and checks, by brute force, that it never rules out a
box that holds a partner passing D2 and D3 as the kernels evaluate them (the operation
order of `doublet_pass`), outward and inward, on random and on boundary-hugging pairs;
and that on the detector's own layers it does rule out the boxes it should (a hit at the
middle of barrel layer 2 cannot reach the first disk), so the test is not vacuous.
"""

import numpy as np

f32 = np.float32


def reachable(cuts, r, z, rlo, rhi, zlo, zhi, outward):
    """The kernels' test, float32, elementwise."""
    r, z, rlo, rhi, zlo, zhi = (np.asarray(v, f32) for v in (r, z, rlo, rhi, zlo, zhi))
    z0max, cot = f32(cuts["z0max"]), f32(cuts["cotmax"])
    if outward:
        d0, d1, e0, e1 = np.maximum(rlo - r, f32(0)), rhi - r, zlo - z, zhi - z
    else:
        d0, d1, e0, e1 = np.maximum(r - rhi, f32(0)), r - rlo, z - zhi, z - zlo
    lo = np.maximum((z - z0max) / r, -cot)
    hi = np.minimum((z + z0max) / r, cot)
    slo = lo - f32(1e-3) * (f32(1) + np.abs(lo))
    shi = hi + f32(1e-3) * (f32(1) + np.abs(hi))
    e0 = e0 - f32(1e-3)
    e1 = e1 + f32(1e-3)
    below = np.where(e1 >= 0, e1 < slo * d0, e1 < slo * d1)
    above = np.where(e0 <= 0, e0 > shi * d0, e0 > shi * d1)
    keep = ~(d1 > 0) | ~(r > 0)
    return keep | ~(below | above)


def d2_d3(cuts, ri, zi, ro, zo):
    """D0, D2 and D3 of `doublet_pass` in float32 (inner hit i, outer hit o)."""
    z0max, cot = f32(cuts["z0max"]), f32(cuts["cotmax"])
    dr, dz = ro - ri, zo - zi
    return (dr > 0) & (np.abs(zi * dr - ri * dz) <= z0max * dr) & (np.abs(dz) <= cot * dr)


def _pairs(rng, n, hug):
    ri = rng.uniform(1.0, 40.0, n).astype(f32)
    ro = (ri + rng.uniform(1e-3, 30.0, n)).astype(f32)
    zi = rng.uniform(-60.0, 60.0, n).astype(f32)
    if hug:
        # partners on the edges of D2 (z0 = +-z0max) and of D3 (|slope| = cotmax)
        z0 = rng.choice([-20.0, 20.0], n) * (1 + rng.normal(0, 1e-6, n))
        s = (zi - z0) / ri
        s = np.where(rng.random(n) < 0.3, rng.choice([-1, 1], n) * 6.6947, s)
        zo = (zi + s * (ro - ri)).astype(f32)
    else:
        zo = (zi + rng.uniform(-8, 8, n) * (ro - ri)).astype(f32)
    return ri, zi, ro, zo


def _boxes_around(rng, r, z, n):
    """Degenerate boxes at the partner and boxes that contain it."""
    tight = rng.random(n) < 0.5
    a = np.where(tight, 0, rng.uniform(0, 5, n)).astype(f32)
    b = np.where(tight, 0, rng.uniform(0, 5, n)).astype(f32)
    c = np.where(tight, 0, rng.uniform(0, 10, n)).astype(f32)
    d = np.where(tight, 0, rng.uniform(0, 10, n)).astype(f32)
    return r - a, r + b, z - c, z + d


def test_never_rules_out_a_passing_partner(cuts):
    rng = np.random.default_rng(2025)
    for hug in (False, True):
        ri, zi, ro, zo = _pairs(rng, 400_000, hug)
        ok = d2_d3(cuts, ri, zi, ro, zo)
        assert ok.sum() > 50_000
        ri, zi, ro, zo = ri[ok], zi[ok], ro[ok], zo[ok]
        # forward search: the inner hit looks outward at a box holding the outer hit
        rlo, rhi, zlo, zhi = _boxes_around(rng, ro, zo, len(ro))
        assert reachable(cuts, ri, zi, rlo, rhi, zlo, zhi, True).all()
        # reverse search: the outer hit looks inward at a box holding the inner hit
        rlo, rhi, zlo, zhi = _boxes_around(rng, ri, zi, len(ri))
        assert reachable(cuts, ro, zo, rlo, rhi, zlo, zhi, False).all()


def test_rules_out_unreachable_layers(cuts):
    # barrel layer 2 (r = 10.9) at z = 0 and the first disk (z = 29.1, r 4.5..16): a cell
    # would need slope >= 29.1 / 5.1, beyond z0max / r = 1.83
    assert not reachable(cuts, 10.9, 0.0, 4.5, 16.0, 29.1, 29.1, True)
    assert not reachable(cuts, 10.9, 0.0, 4.5, 16.0, -29.1, -29.1, True)
    # inward from that disk at r = 12, z = 29.1 to layer 2's box (r 10.9, |z| <= 27):
    # slopes from 2.1 / 1.1 up, allowed up to (29.1 + 20) / 12, so reachable
    assert reachable(cuts, 12.0, 29.1, 10.9, 10.9, -27.0, 27.0, False)
    # a box at or beyond the hit's own radius is left to D0
    assert reachable(cuts, 5.0, 29.1, 10.9, 10.9, -27.0, 27.0, False)
    # the beam line: a hit at z = 25 on layer 0 reaches the + disk, not the - disk
    assert reachable(cuts, 2.9, 25.0, 4.5, 16.0, 29.1, 29.1, True)
    assert not reachable(cuts, 2.9, 25.0, 4.5, 16.0, -29.1, -29.1, True)


def test_detector_skip_share(cuts):
    """On simulated PU200 hits, the layer pairs of the default table: a sizeable share of
    (hit, layer) windows is ruled out, and no ruled-out window holds a cell."""
    import sim
    import paper_2501_05520_gb300 as pt
    ev = sim.generate(sim.PU200, 3000)
    x, y, z = (np.asarray(v, f32) for v in (ev.x, ev.y, ev.z))
    r = np.sqrt(x * x + y * y).astype(f32)
    lay = np.asarray(ev.layer)
    skipped = total = 0
    for Li, Lo in pt.DEFAULT_PAIRS:
        I, O = np.where(lay == Li)[0], np.where(lay == Lo)[0]
        box = (r[O].min(), r[O].max(), z[O].min(), z[O].max())
        keep = reachable(cuts, r[I], z[I], *box, True)
        total += len(I)
        skipped += int((~keep).sum())
        # the ruled-out inner hits have no partner in O passing D2 and D3
        for i in I[~keep][:200]:
            assert not d2_d3(cuts, r[i], z[i], r[O], z[O]).any()
    assert skipped > 0.1 * total, (skipped, total)
