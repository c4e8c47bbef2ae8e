"""Pins of the broken-line refit oracle (oracle/brokenline.py) and of the generator's
multiple scattering: exact helices recovered from a perturbed reference, a planted
kink found at its plane, triplets on their circumcircle, pulls and chi2 of scattered
tracks, and the stepwise propagator against the closed-form crossings."""

import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import brokenline as bl
from sim import events as E


def helix(kappa, phi0, d0, cot, z0, s):
    """Closed-form helix at transverse arc lengths s from its closest approach
    d0 (sin phi0, -cos phi0): direction phi0 + kappa s, z = z0 + cot s."""
    psi = phi0 + kappa * s
    x = d0 * math.sin(phi0) + (np.sin(psi) - math.sin(phi0)) / kappa
    y = -d0 * math.cos(phi0) - (np.cos(psi) - math.cos(phi0)) / kappa
    return x, y, z0 + cot * s


CASES = [  # kappa, phi0, d0, cot, z0, arc lengths, layers
    (0.0123, 0.7, 0.003, 0.45, 1.3, [3.0, 7.1, 11.2, 16.4], [0, 1, 2, 3]),
    (-0.0123, 0.7, 0.003, 0.45, 1.3, [3.0, 7.1, 11.2, 16.4, 20.0], [0, 1, 2, 3, 4]),
    (0.031, -2.9, -0.02, -1.7, -4.0, [2.9, 7.0, 17.0, 23.0], [0, 1, 7, 8]),
    (-0.0009, 3.1, 0.0, 0.05, 0.2, [2.9, 6.8, 10.9, 16.0], [0, 1, 2, 3]),
    (0.02, 1.5, 0.01, 3.0, 2.0, [4.0, 9.0, 13.0, 17.0, 21.0, 25.0], [0, 4, 5, 6, 6, 6]),
]


@pytest.mark.parametrize("case", CASES)
def test_exact_helix_from_perturbed_reference(case):
    """Noiseless hits of a helix and a reference off by 1e-3 in curvature, 2e-4 rad,
    3 um, 1e-3 in slope and 20 um: the refit lands on the helix up to second-order
    terms (below 5e-7 relative in curvature and 1e-5 cm in z0 on these arcs of up to
    0.7 rad), while a sign, index or coefficient slip leaves first-order errors of a
    per cent or more of the perturbation."""
    k, phi0, d0, cot, z0, s, lay = case
    x, y, z = helix(k, phi0, d0, cot, z0, np.asarray(s))
    ref = np.array([k * (1 + 1e-3), phi0 + 2e-4, d0 + 3e-4, cot + 1e-3, z0 + 2e-3])
    out = bl.refit(x, y, z, np.asarray(lay), ref, 0.02, 0.03)
    assert abs(out[0] - k) <= 1e-6 * abs(k)
    assert abs(math.remainder(out[1] - phi0, 2 * math.pi)) <= 2e-7
    assert abs(out[2] - d0) <= 3e-7
    assert abs(out[3] - cot) <= 1e-6
    assert abs(out[4] - z0) <= 2e-5
    assert out[6] < 1e-6 and out[7] < 1e-6
    assert out[8] == -math.copysign(1.0, k)
    assert out[5] == pytest.approx(0.299792458 * 3.8 / (100 * abs(k)), rel=1e-5)


def test_planted_kink_is_found_at_its_plane():
    """Two arcs of one helix joined at the second plane by a turn of 1e-3 rad in the
    transverse direction and 2e-3 in dz/ds; material only at that plane (a disk code)
    and precise hits: the refit puts the whole kink there and keeps the curvature."""
    k, phi0, cot, z0 = 0.01, 0.3, 0.2, 0.5
    xa, ya, za = helix(k, phi0, 0.0, cot, z0, np.array([3.0, 7.0]))
    alpha, gam = 1e-3, 2e-3
    psi2 = phi0 + k * 7.0 + alpha
    ss = np.cumsum([4.1, 5.0, 4.5])
    xb = xa[1] + (np.sin(psi2 + k * ss) - math.sin(psi2)) / k
    yb = ya[1] - (np.cos(psi2 + k * ss) - math.cos(psi2)) / k
    zb = za[1] + (cot + gam) * ss
    x, y, z = np.r_[xa, xb], np.r_[ya, yb], np.r_[za, zb]
    lay = np.array([0, 4, 1, 2, 3])
    ref = oracle.fit_hits(x, y, z)
    out, d = bl.refit(x, y, z, lay, ref, 1e-9, 0.05, sigma_t=1e-7, sigma_l=1e-7, full=True)
    # the planted turns, to first order in the offsets (a few 1e-6 relative)
    assert d["beta"][0] == pytest.approx(alpha, rel=1e-4)
    assert np.all(np.abs(d["beta"][1:]) < 1e-6 * alpha)
    assert d["gamma"][0] == pytest.approx(gam, rel=1e-4)
    assert np.all(np.abs(d["gamma"][1:]) < 1e-4 * gam)
    assert out[0] == pytest.approx(k, rel=1e-6)
    assert abs(math.remainder(out[1] - phi0, 2 * math.pi)) < 1e-8
    assert abs(out[3] - cot) < 1e-6 and abs(out[4] - z0) < 1e-6


@pytest.mark.parametrize("seed", range(6))
def test_triplet_lies_on_its_circumcircle(seed):
    """Three hits fix a circle: from a perturbed reference the refit returns the
    curvature of the circle through them (the closed form 2 (b-a) x (c-b) /
    (|b-a| |c-b| |c-a|)) with zero transverse chi2."""
    rng = np.random.default_rng(seed)
    r = np.array([2.9, 6.8, 10.9]) + rng.uniform(0, 0.5, 3)
    ang = rng.uniform(-3, 3) + np.cumsum(rng.uniform(-0.03, 0.03, 3))
    x, y = r * np.cos(ang), r * np.sin(ang)
    z = rng.uniform(-5, 5) + r * rng.uniform(-2, 2)
    a, b, c = np.c_[x, y]
    cross = (b - a)[0] * (c - b)[1] - (b - a)[1] * (c - b)[0]
    k3 = 2 * cross / (np.linalg.norm(b - a) * np.linalg.norm(c - b) * np.linalg.norm(c - a))
    ref = oracle.fit_hits(x, y, z)
    ref[0] *= 1 + 1e-3
    ref[1] += 1e-4
    out = bl.refit(x, y, z, np.array([0, 1, 2]), ref, 0.02, 0.02)
    assert out[0] == pytest.approx(k3, rel=1e-6)
    assert out[6] < 1e-12


def _scattered_tracks(seed, n, pt_lo, pt_hi, eta_max, x0):
    rng = np.random.default_rng(seed)
    pt = rng.uniform(pt_lo, pt_hi, n)
    eta = rng.uniform(-eta_max, eta_max, n)
    p = dict(pt=pt, eta=eta, phi0=rng.uniform(0, 2 * np.pi, n),
             q=np.where(rng.random(n) < 0.5, -1.0, 1.0), z0=rng.normal(0, 5, n),
             R=pt / (E.C_LIGHT * E.BFIELD_T) * 100.0)
    pid, lay, xt, yt, zt, step = E._crossings_ms(rng, p, eta_max <= 1.0, x0, x0)
    xs, ys, zs = E._smear(rng, lay, xt, yt, zt)
    return p, pid, lay, xs, ys, zs, step


@pytest.mark.parametrize("pt_lo,pt_hi,eta_max", [(0.5, 0.8, 1.0), (0.6, 1.0, 2.4)])
def test_pulls_and_chi2_of_scattered_tracks(pt_lo, pt_hi, eta_max):
    """Smeared tracks that scatter in 2 % X0 per layer: curvature pulls against the
    generated value and slope pulls (fit variance plus the unmeasured scattering at
    the first plane) have mean 0 and width 1, and chi2 per degree of freedom is 1 in
    both planes (3000 tracks: 3 sigma is 0.055 on a mean, 0.04 on a width and 0.08 on
    chi2/ndf of quadruplets).  The circle fit's chi2, blind to scattering, is not."""
    x0 = 0.02
    p, pid, lay, xs, ys, zs, step = _scattered_tracks(11, 3000, pt_lo, pt_hi, eta_max, x0)
    pk, pc, ct, cl, cc, nt, nl = [], [], [], [], [], [], []
    for i in range(p["pt"].size):
        m = np.flatnonzero(pid == i)
        if m.size < 3:
            continue
        m = m[np.argsort(step[m])]
        ref = oracle.fit_hits(xs[m], ys[m], zs[m])
        out, d = bl.refit(xs[m], ys[m], zs[m], lay[m], ref, x0, x0, full=True)
        pk.append((out[0] + p["q"][i] / p["R"][i]) / math.sqrt(d["var_kappa"]))
        pc.append((out[3] - math.sinh(p["eta"][i])) / math.sqrt(d["var_cot"] + d["var_l"][0]))
        ct.append(out[6])
        cl.append(out[7])
        cc.append(ref[6])
        nt.append(m.size - 3)
        nl.append(m.size - 2)
    pk, pc = np.asarray(pk), np.asarray(pc)
    assert pk.size > 2900
    assert abs(pk.mean()) < 0.06 and 0.95 < pk.std() < 1.05
    assert abs(pc.mean()) < 0.06 and 0.95 < pc.std() < 1.05
    assert 0.9 < sum(ct) / sum(nt) < 1.1
    assert 0.9 < sum(cl) / sum(nl) < 1.1
    assert sum(cc) / sum(nt) > 5.0


def test_propagator_without_scattering_matches_closed_form():
    """The surface-by-surface propagator with negligible material finds the same
    crossings as the closed-form helix intersections."""
    cfg = dataclasses.replace(E.PU50, n_particles=2000, smear=False, noise_frac=0.0)
    p = E._draw_particles(np.random.default_rng(5), cfg, 2000)
    a = E._crossings(p, False)
    b = E._crossings_ms(np.random.default_rng(1), p, False, 1e-300, 1e-300)
    ia, ib = np.lexsort((a[1], a[0])), np.lexsort((b[1], b[0]))
    assert np.array_equal(a[0][ia], b[0][ib]) and np.array_equal(a[1][ia], b[1][ib])
    for u, v in zip(a[2:5], b[2:5]):
        assert np.max(np.abs(u[ia] - v[ib])) < 1e-9


def test_material_off_leaves_events_unchanged():
    """Configurations without material keep the closed-form generator."""
    a = E.generate(E.PU50, 2000)
    b = E.generate(dataclasses.replace(E.PU50, x0_barrel=0.0, x0_disk=0.0), 2000)
    assert np.array_equal(a.x64, b.x64) and np.array_equal(a.pid, b.pid)
    c = E.generate(dataclasses.replace(E.PU50, x0_barrel=0.02, x0_disk=0.02), 2000)
    assert c.n_hits > 0.95 * a.n_hits and not np.array_equal(a.x64[:100], c.x64[:100])


def test_iterated_refit_is_a_fixed_point():
    """[B7] After the passes stop, one more pass from the result changes the curvature
    by far less than the stopping threshold (on a forward sample where the first pass
    moves it by per cents)."""
    x0 = 0.02
    p, pid, lay, xs, ys, zs, step = _scattered_tracks(12, 600, 0.5, 0.9, 2.4, x0)
    worst_first, worst_after = 0.0, 0.0
    for i in range(p["pt"].size):
        m = np.flatnonzero(pid == i)
        if m.size < 3:
            continue
        m = m[np.argsort(step[m])]
        ref = oracle.fit_hits(xs[m], ys[m], zs[m])
        one = bl.refit(xs[m], ys[m], zs[m], lay[m], ref, x0, x0)
        it = bl.refit_iterated(xs[m], ys[m], zs[m], lay[m], ref, x0, x0)
        again = bl.refit(xs[m], ys[m], zs[m], lay[m], it, x0, x0)
        worst_first = max(worst_first, abs(one[0] - ref[0]) / abs(ref[0]))
        worst_after = max(worst_after, abs(again[0] - it[0]) / abs(it[0]))
    assert worst_first > 0.02
    assert worst_after < 1e-4


def _arc_tangents(p0, p1, R, q):
    """Unit tangents at p0 and p1 of the minor arc of radius R from p0 to p1, turning
    clockwise for q > 0 and counter-clockwise for q < 0."""
    u = p1 - p0
    lu = np.hypot(u[0], u[1])
    m = 0.5 * (p0 + p1)
    b = math.sqrt(max(R * R - 0.25 * lu * lu, 0.0))
    right = np.array([u[1], -u[0]]) / lu
    c = m + (b if q > 0 else -b) * right

    def tangent(pt):
        r = pt - c
        t = np.array([r[1], -r[0]]) if q > 0 else np.array([-r[1], r[0]])
        return t / np.hypot(t[0], t[1])

    return tangent(p0), tangent(p1)


def test_generator_scattering_follows_highland():
    """Noiseless barrel tracks at eta = 0 (all scattering in the transverse direction
    shows as a turn of the arc): the turn at each interior layer, measured from the arcs
    of known radius through consecutive hits, divided by the Highland width for that
    crossing (13.6 MeV / p sqrt(t)(1 + 0.038 ln t), t = x0 / cos(incidence)) has mean 0
    and width 1 (2 x 2000 turns: 3 sigma is 0.05 on the width)."""
    x0, n = 0.03, 2000
    rng = np.random.default_rng(21)
    pt_ = np.full(n, 0.8)
    p = dict(pt=pt_, eta=np.zeros(n), phi0=rng.uniform(0, 2 * np.pi, n),
             q=np.where(rng.random(n) < 0.5, -1.0, 1.0), z0=np.zeros(n),
             R=pt_ / (E.C_LIGHT * E.BFIELD_T) * 100.0)
    pid, lay, x, y, z, step = E._crossings_ms(rng, p, True, x0, x0)
    pulls = []
    for i in range(n):
        m = np.flatnonzero(pid == i)
        m = m[np.argsort(step[m])]
        assert lay[m].tolist() == [0, 1, 2, 3]
        pts = [np.array([x[k], y[k]]) for k in m]
        R, q = p["R"][i], p["q"][i]
        for j in (1, 2):
            _, t_in = _arc_tangents(pts[j - 1], pts[j], R, q)
            t_out, _ = _arc_tangents(pts[j], pts[j + 1], R, q)
            turn = math.atan2(t_in[0] * t_out[1] - t_in[1] * t_out[0], t_in @ t_out)
            cos_inc = abs(t_in @ pts[j]) / np.hypot(*pts[j])
            t = x0 / cos_inc
            th0 = 0.0136 / 0.8 * math.sqrt(t) * (1.0 + 0.038 * math.log(t))
            pulls.append(math.tan(turn) / th0)
    pulls = np.asarray(pulls)
    assert abs(pulls.mean()) < 0.07 and 0.95 < pulls.std() < 1.05


def test_refit_improves_z0_and_slope_resolution():
    """What the refit is for: on tracks that scatter in 2 % X0 per layer its z0 and
    cot(theta) scatter less about the generated values than those of the circle + line
    fit (low-momentum barrel tracks: z0 about 170 -> 105 um)."""
    p, pid, lay, xs, ys, zs, step = _scattered_tracks(31, 1500, 0.5, 0.8, 1.0, 0.02)
    dz_c, dz_b, dc_c, dc_b = [], [], [], []
    for i in range(p["pt"].size):
        m = np.flatnonzero(pid == i)
        if m.size < 4:
            continue
        m = m[np.argsort(step[m])]
        ref = oracle.fit_hits(xs[m], ys[m], zs[m])
        out = bl.refit_iterated(xs[m], ys[m], zs[m], lay[m], ref, 0.02, 0.02)
        dz_c.append(ref[4] - p["z0"][i])
        dz_b.append(out[4] - p["z0"][i])
        dc_c.append(ref[3] - math.sinh(p["eta"][i]))
        dc_b.append(out[3] - math.sinh(p["eta"][i]))
    rms = lambda a: float(np.sqrt(np.mean(np.square(a))))  # noqa: E731
    assert rms(dz_b) < 0.75 * rms(dz_c)
    assert rms(dc_b) < 0.9 * rms(dc_c)
