"""Pins of the CPU oracle against facts fixed by geometry, closed forms and brute force.

Each check uses a formulation of the cut's meaning that differs from the oracle's
division-free float32 form (polar angles, the inscribed-angle theorem, explicit circle
centres, line extrapolation), so a dropped term, a wrong sign or a swapped operand in
the oracle fails here.  Decisions within 1e-4 relative of a threshold are skipped
(float32 vs float64 rounding), and their number is bounded.
"""

import math

import networkx as nx
import numpy as np
import pytest

import oracle
import sim
from sim import truth

MARGIN = 1e-4


def _tiny_event(seed, n_particles=40, noise=0.3):
    cfg = sim.GenConfig(n_particles, "inv_pt_uniform", 2.5, False, noise)
    return sim.generate(cfg, seed)


def _f64(e):
    x = e.x.astype(np.float64)
    y = e.y.astype(np.float64)
    z = e.z.astype(np.float64)
    return x, y, z, np.hypot(x, y)


def _clear(value, thr):
    """True where value is at least MARGIN (relative) away from thr."""
    return np.abs(value - thr) > MARGIN * np.maximum(np.abs(value), np.abs(thr))


def test_doublets_match_geometric_definition(cuts):
    """Every hit pair on an allowed layer pair: accepted iff outward, within 90 degrees in
    azimuth, the circle through beam spot and both hits has curvature <= kmax (inscribed
    angle theorem), |z| of the r-z line at r=0 <= z0max and |dz/dr| <= cotmax."""
    n_checked = n_skipped = 0
    for seed in range(20):
        e = _tiny_event(100 + seed)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
        got = set(zip(res["cell_inner"].tolist(), res["cell_outer"].tolist()))
        x, y, z, r = _f64(e)
        phi = np.arctan2(y, x)
        exp, amb = set(), set()
        n_pairs = 0
        for li, lo in truth.LAYER_PAIRS:
            I = np.flatnonzero(e.layer == li)
            O = np.flatnonzero(e.layer == lo)
            if I.size == 0 or O.size == 0:
                continue
            i, o = np.meshgrid(I, O, indexing="ij")
            i, o = i.ravel(), o.ravel()
            n_pairs += i.size
            dphi = np.angle(np.exp(1j * (phi[o] - phi[i])))
            chord = np.hypot(x[o] - x[i], y[o] - y[i])
            kappa = 2.0 * np.abs(np.sin(dphi)) / chord
            dr = r[o] - r[i]
            with np.errstate(divide="ignore", invalid="ignore"):
                slope = (z[o] - z[i]) / dr
                z0 = z[i] - r[i] * slope
            ok = ((dr > 0) & (np.abs(dphi) < np.pi / 2) & (kappa <= cuts["kmax"])
                  & (np.abs(z0) <= cuts["z0max"]) & (np.abs(slope) <= cuts["cotmax"]))
            clear = (_clear(r[o], r[i]) & _clear(np.abs(dphi), np.pi / 2)
                     & _clear(kappa, cuts["kmax"]) & _clear(np.abs(z0), cuts["z0max"])
                     & _clear(np.abs(slope), cuts["cotmax"]))
            for a, b, k, c in zip(i.tolist(), o.tolist(), ok.tolist(), clear.tolist()):
                if not c:
                    amb.add((a, b))
                elif k:
                    exp.add((a, b))
        n_checked += n_pairs - len(amb)
        n_skipped += len(amb)
        assert len(exp) > 50
        assert (got - amb) == exp, f"seed {seed}"
    assert n_skipped < 1e-3 * n_checked


def _circle(p0, p1, p2):
    """Circumcentre and radius by solving the two perpendicular-bisector equations."""
    A = 2.0 * np.array([p1 - p0, p2 - p0])
    b = np.array([p1 @ p1 - p0 @ p0, p2 @ p2 - p0 @ p0])
    c = np.linalg.solve(A, b)
    return c, float(np.hypot(*(p0 - c)))


def test_links_match_geometric_definition(cuts):
    """Every pair of oracle cells sharing a hit: linked iff the middle hit lies within
    rz0 + rz1 |z2-z0|/(r2-r0) in z of the chord through the outer hits (r-z plane),
    the circle through the three hits has curvature <= kmax (inscribed angle at the
    middle hit), and that circle passes within dcamax of the beam spot.  The link
    quality equals that distance."""
    n_checked = n_skipped = 0
    for seed in range(20):
        e = _tiny_event(200 + seed, n_particles=60, noise=0.5)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
        ci, co = res["cell_inner"], res["cell_outer"]
        got = {(int(a), int(b)): float(q)
               for a, b, q in zip(res["link_a"], res["link_b"], res["link_q"])}
        x, y, z, r = _f64(e)
        P = np.stack([x, y], 1)
        for a in range(ci.size):
            for b in np.flatnonzero(ci == co[a]).tolist():
                h0, h1, h2 = int(ci[a]), int(co[a]), int(co[b])
                dz_mid = z[h1] - (z[h0] + (z[h2] - z[h0]) * (r[h1] - r[h0]) / (r[h2] - r[h0]))
                tol = cuts["rz0"] + cuts["rz1"] * abs(z[h2] - z[h0]) / (r[h2] - r[h0])
                v0, v2 = P[h0] - P[h1], P[h2] - P[h1]
                ang = math.atan2(v0[0] * v2[1] - v0[1] * v2[0], v0 @ v2)
                kappa = 2.0 * abs(math.sin(ang)) / float(np.hypot(*(P[h2] - P[h0])))
                c, R = _circle(P[h0], P[h1], P[h2])
                dca = abs(float(np.hypot(*c)) - R)
                dmax = cuts["dca_b0"] if e.layer[h0] == 0 else cuts["dca_other"]
                ok = abs(dz_mid) <= tol and kappa <= cuts["kmax"] and dca <= dmax
                clear = (_clear(abs(dz_mid), tol) and _clear(kappa, cuts["kmax"])
                         and _clear(dca, dmax))
                if not clear:
                    n_skipped += 1
                    continue
                n_checked += 1
                assert ((a, b) in got) == ok, (seed, a, b)
                if ok:
                    assert got[(a, b)] == pytest.approx(dca, rel=1e-3, abs=1e-5)
    assert n_checked > 2000
    assert n_skipped < 0.01 * n_checked


def test_link_quality_is_line_distance_for_collinear_hits():
    """Collinear hits: the circle degenerates to a line and the quality is the distance
    from the beam spot to that line (here x - 2y + 2 = 0, distance 2/sqrt(5))."""
    wide = dict(kmax=1.0, z0max=100.0, cotmax=100.0, rz0=1.0, rz1=1.0, dca_b0=5.0,
                dca_other=5.0)
    ok, near, q = oracle.link_ok(wide, (2.0, 2.0, 0.0), 1, (4.0, 3.0, 0.0), (6.0, 4.0, 0.0))
    assert ok and not near
    assert q == pytest.approx(2.0 / math.sqrt(5.0), rel=1e-6)


def test_threshold_equality_is_accepted_and_logged():
    """A cut variable exactly on its threshold passes (<=) and is logged as near."""
    cot = float(np.float32(6.694732189178467))
    zo = float(np.float32(np.float32(cot) * np.float32(4.0)))
    c = dict(kmax=1.0, z0max=1000.0, cotmax=cot, rz0=0.02, rz1=0.01, dca_b0=0.05,
             dca_other=0.2)
    ok, near = oracle.doublet_ok(c, (3.0, 0.0, 0.0), (7.0, 0.0, zo))
    assert ok and near
    ok, near = oracle.doublet_ok(c, (3.0, 0.0, 0.0), (7.0, 0.0, float(np.nextafter(
        np.float32(zo), np.float32(100)))))
    assert not ok and near


def _draw_helix(rng, barrel_only):
    eta_max = 1.0 if barrel_only else 2.5
    return dict(pt=1.0 / rng.uniform(0.1, 2.0), eta=rng.uniform(-eta_max, eta_max),
                phi0=rng.uniform(-math.pi, math.pi), q=float(rng.choice([-1.0, 1.0])),
                z0=float(np.clip(rng.normal(0, 5), -15, 15)))


@pytest.mark.parametrize("barrel_only", [True, False])
def test_single_noiseless_helix_gives_its_chain(cuts, barrel_only):
    """A lone noiseless helix gives exactly one ntuplet: its hits on the longest chain of
    allowed layer pairs (inner to outer), when that chain has >= 3 hits."""
    rng = np.random.default_rng(7 + barrel_only)
    n_with = 0
    for k in range(300):
        p = _draw_helix(rng, barrel_only)
        e = sim.single_helix(k, p["pt"], p["eta"], p["phi0"], p["q"], p["z0"], barrel_only)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
        chain = truth.particle_chains(e.pid, e.layer)[0]["chain"] if e.n_hits else np.array([])
        sv = oracle.survivors_hits(res)
        if chain.size >= 3:
            n_with += 1
            assert sv.shape[0] == 1, (k, p)
            assert sv[0][: chain.size].tolist() == chain.tolist()
            assert (sv[0][chain.size:] == -1).all()
        else:
            assert sv.shape[0] == 0
    assert n_with > 200


def test_fit_closed_form_noiseless_helix():
    """Float64 noiseless crossings: curvature = -charge/R, phi0, cot(theta) = sinh(eta),
    z0 and pT as generated, d0 = 0, all to 1e-6 relative (floors 1 cm, 1 rad)."""
    rng = np.random.default_rng(11)
    n = 0
    for k in range(300):
        p = _draw_helix(rng, barrel_only=False)
        e = sim.single_helix(k, p["pt"], p["eta"], p["phi0"], p["q"], p["z0"], False)
        ch = truth.particle_chains(e.pid, e.layer)
        if not ch or ch[0]["hits"].size < 3:
            continue
        h = ch[0]["hits"]
        f = oracle.fit_hits(e.xt[h], e.yt[h], e.zt[h])
        R = e.particles["R"][0]
        assert f[0] == pytest.approx(-p["q"] / R, rel=1e-6)
        assert f[8] == p["q"]
        dphi = math.remainder(f[1] - p["phi0"], 2 * math.pi)
        assert abs(dphi) <= 1e-6
        assert abs(f[2]) <= 1e-6
        assert f[3] == pytest.approx(math.sinh(p["eta"]), rel=1e-6, abs=1e-6)
        assert abs(f[4] - p["z0"]) <= 1e-6 * max(abs(p["z0"]), 1.0)
        assert f[5] == pytest.approx(p["pt"], rel=1e-6)
        assert f[6] < 1e-6 and f[7] < 1e-6
        n += 1
    assert n > 200


def test_fit_triplet_equals_circumcircle():
    """Three float32 hits: the circle fit is exact, so |kappa| = 1/R of the circumcircle,
    |d0| = | |centre| - R |, and kappa > 0 iff the hits turn counter-clockwise."""
    n = 0
    for seed in range(5):
        e = sim.generate(sim.PU50, 9000 + seed, n_particles=200)
        x, y, z, _ = _f64(e)
        P = np.stack([x, y], 1)
        for h0, h1, h2 in truth.true_triplets(e.pid, e.layer):
            c, R = _circle(P[h0], P[h1], P[h2])
            f = oracle.fit_hits(x[[h0, h1, h2]], y[[h0, h1, h2]], z[[h0, h1, h2]])
            assert abs(f[0]) == pytest.approx(1.0 / R, rel=1e-9)
            assert abs(f[2]) == pytest.approx(abs(float(np.hypot(*c)) - R), rel=1e-6, abs=1e-9)
            a, b = P[h1] - P[h0], P[h2] - P[h0]
            assert (f[0] > 0) == (a[0] * b[1] - a[1] * b[0] > 0)
            n += 1
    assert n > 500


def _helix_at_pca(rng, b, sign, kappa, cot, z0, arcs):
    """Float64 points of a helix built from its point of closest approach P to the beam
    line: P at distance b in a random direction, the transverse direction t at P
    perpendicular to P (turned left of P for sign = +1, right for -1), the circle of
    signed curvature kappa tangent to t at P (centre on the left of t for kappa > 0), and
    the points at the given transverse arc lengths from P with z = z0 + cot * s.
    Returns the points with the signed impact parameter P x t and the direction of t,
    both computed from the construction rather than from any fit convention."""
    beta = rng.uniform(-math.pi, math.pi)
    P = b * np.array([math.cos(beta), math.sin(beta)])
    t = sign * np.array([-math.sin(beta), math.cos(beta)])
    left = np.array([-t[1], t[0]])
    C = P + left / kappa
    v = P - C
    ang = kappa * np.asarray(arcs)
    x = C[0] + np.cos(ang) * v[0] - np.sin(ang) * v[1]
    y = C[1] + np.sin(ang) * v[0] + np.cos(ang) * v[1]
    z = z0 + cot * np.asarray(arcs)
    d0 = float(P[0] * t[1] - P[1] * t[0])
    return x, y, z, d0, math.atan2(t[1], t[0]), C


def test_fit_signed_impact_parameter_displaced_helices():
    """Noiseless helices whose closest approach to the beam line lies 0.01-0.5 cm from it,
    on either side, for both charges: the fit returns the construction's signed d0 = P x t
    (the z component of the closest-approach point crossed with the unit direction of
    travel there), its direction phi0, curvature, cot(theta) and z0 at that point, to
    1e-6 relative.  A flipped d0 sign or a closest-approach point taken on the wrong side
    of the circle fails on half of the cases."""
    rng = np.random.default_rng(23)
    signs = set()
    for k in range(2000):
        b = rng.uniform(0.01, 0.5)
        side = float(rng.choice([-1.0, 1.0]))
        q = float(rng.choice([-1.0, 1.0]))
        R = 100.0 / rng.uniform(0.1, 2.0) / (0.299792458 * 3.8)
        kappa = -q / R
        cot = math.sinh(rng.uniform(-2.5, 2.5))
        z0 = rng.normal(0.0, 5.0)
        n = int(rng.integers(3, 7))
        arcs = np.sort(rng.uniform(2.5, 18.0, n))
        x, y, z, d0, phi0, C = _helix_at_pca(rng, b, side, kappa, cot, z0, arcs)
        assert abs(abs(d0) - b) <= 1e-12 and abs(float(np.hypot(*C)) - (R - d0 * np.sign(kappa))) < 1e-9 * R
        f = oracle.fit_hits(x, y, z)
        assert f[0] == pytest.approx(kappa, rel=1e-6), k
        assert f[2] == pytest.approx(d0, rel=1e-6), k
        assert abs(math.remainder(f[1] - phi0, 2 * math.pi)) <= 1e-6, k
        assert f[3] == pytest.approx(cot, rel=1e-6, abs=1e-6), k
        assert abs(f[4] - z0) <= 1e-6 * max(abs(z0), 1.0), k
        assert f[8] == q
        signs.add((np.sign(d0), q))
    assert len(signs) == 4


def test_fit_chi2_per_degree_of_freedom_is_one():
    """Hits moved off an exact helix along the circle's normal by N(0, 10 um) and in z by
    N(0, 20 um), the resolutions the fit divides by: summed over 3000 tracks of 4-6 hits,
    chi2_circle / (n - 3) and chi2_line / (n - 2) are 1 within five standard deviations
    of a chi-square mean, sqrt(2 / total ndf).  A wrong resolution, a missing factor in
    the residual or a wrong degree-of-freedom count fails."""
    rng = np.random.default_rng(31)
    sig_rphi, sig_z = 10e-4, 20e-4
    c2c = c2l = ndf_c = ndf_l = 0.0
    for k in range(3000):
        q = float(rng.choice([-1.0, 1.0]))
        R = 100.0 / rng.uniform(0.1, 2.0) / (0.299792458 * 3.8)
        cot = math.sinh(rng.uniform(-2.0, 2.0))
        n = int(rng.integers(4, 7))
        arcs = np.sort(rng.uniform(2.5, 18.0, n))
        x, y, z, _, _, C = _helix_at_pca(rng, rng.uniform(0.0, 0.1), float(rng.choice([-1.0, 1.0])),
                                         -q / R, cot, rng.normal(0.0, 5.0), arcs)
        rad = np.hypot(x - C[0], y - C[1])
        move = rng.normal(0.0, sig_rphi, n)
        x = x + move * (x - C[0]) / rad
        y = y + move * (y - C[1]) / rad
        z = z + rng.normal(0.0, sig_z, n)
        f = oracle.fit_hits(x, y, z)
        c2c += f[6]
        c2l += f[7]
        ndf_c += n - 3
        ndf_l += n - 2
    assert abs(c2c / ndf_c - 1.0) <= 5.0 * math.sqrt(2.0 / ndf_c), c2c / ndf_c
    assert abs(c2l / ndf_l - 1.0) <= 5.0 * math.sqrt(2.0 / ndf_l), c2l / ndf_l


def test_ntuplets_are_all_maximal_chains(cuts):
    """Ntuplets are exactly the root-to-leaf paths (>= 2 cells) of the link graph, as
    enumerated by networkx; consecutive cells share a hit; the layer sequence follows
    allowed pairs; q is the float32 inner-to-outer sum of the link qualities."""
    allowed = set(truth.LAYER_PAIRS)
    for seed in range(3):
        e = sim.generate(sim.PU50, 2100 + seed, n_particles=600)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
        C = res["cell_inner"].size
        G = nx.DiGraph()
        G.add_nodes_from(range(C))
        lq = {}
        for a, b, q in zip(res["link_a"].tolist(), res["link_b"].tolist(), res["link_q"]):
            G.add_edge(a, b)
            lq[(a, b)] = np.float32(q)
        leaves = [v for v in G if G.out_degree(v) == 0]
        exp = set()
        for root in (v for v in G if G.in_degree(v) == 0 and G.out_degree(v) > 0):
            for path in nx.all_simple_paths(G, root, leaves):
                exp.add(tuple(path))
        got = set()
        for t in range(res["nt_n"].size):
            n = int(res["nt_n"][t])
            cells = res["nt_cells"][t][: n - 1].tolist()
            hits = res["nt_hits"][t][:n].tolist()
            assert 3 <= n <= 6
            assert hits[0] == res["cell_inner"][cells[0]]
            for k, c in enumerate(cells):
                assert res["cell_outer"][c] == hits[k + 1]
            lay = e.layer[hits].tolist()
            assert all((u, v) in allowed for u, v in zip(lay[:-1], lay[1:]))
            q = np.float32(0.0)
            for a, b in zip(cells[:-1], cells[1:]):
                q = np.float32(q + lq[(a, b)])
            assert q == res["nt_q"][t]
            got.add(tuple(cells))
        assert len(got) == res["nt_n"].size
        assert got == exp
        assert len(exp) > 100


def _pack(ntuplets):
    """ntuplets: list of (hits list, cells list, q) -> dedup arrays."""
    T = len(ntuplets)
    hits = np.full((T, 6), -1, np.int32)
    cells = np.full((T, 5), -1, np.int32)
    nh = np.zeros(T, np.int32)
    q = np.zeros(T, np.float32)
    for t, (h, c, qq) in enumerate(ntuplets):
        hits[t, : len(h)] = h
        cells[t, : len(c)] = c
        nh[t] = len(h)
        q[t] = qq
    return hits, cells, nh, q


@pytest.mark.parametrize("case,expected", [
    # two quadruplets sharing cell 1: the smaller q wins
    ([([0, 1, 2, 3], [0, 1, 2], 0.5), ([10, 1, 2, 4], [5, 1, 6], 0.2)], [1]),
    # a quadruplet beats a triplet on a shared cell whatever their q
    ([([0, 1, 2, 3], [0, 1, 2], 9.0), ([1, 2, 7], [1, 8], 0.0)], [0]),
    # equal hits and q: the smaller hit tuple wins
    ([([0, 1, 5], [0, 3], 0.25), ([0, 1, 4], [0, 4], 0.25)], [1]),
    # a triplet sharing only a hit (no cell) with a surviving quadruplet is dropped,
    # an unrelated triplet stays
    ([([0, 1, 2, 3], [0, 1, 2], 0.1), ([20, 21, 3], [9, 10], 0.0), ([30, 31, 32], [11, 12], 0.0)],
     [0, 2]),
    # a triplet sharing a hit with a quadruplet that lost its own cell stays
    # (cell 2 is the hit pair (2, 3), shared by t0 and t1; t1 wins it)
    ([([0, 1, 2, 3], [0, 1, 2], 0.9), ([5, 6, 2, 3], [13, 14, 2], 0.1), ([40, 41, 0], [15, 16], 0.0)],
     [1, 2]),
    # no cascade: t0 beats t1 on cell 1, t1 beats t2 on cell 4; t2 dies although t1 died
    ([([0, 1, 2, 3], [0, 1, 2], 0.1), ([9, 1, 2, 8], [7, 1, 4], 0.2), ([11, 12, 2, 8], [5, 6, 4], 0.3)],
     [0]),
])
def test_dedup_hand_built(case, expected):
    hits, cells, nh, q = _pack(case)
    got = oracle.dedup(hits, cells, nh, q, n_cells=32, n_hits=64)
    assert got.tolist() == expected


def test_dedup_output_is_canonically_ordered(cuts):
    e = sim.generate(sim.PU50, 2200)
    res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
    sv = oracle.survivors_hits(res)
    keys = [tuple(r) for r in sv.tolist()]
    assert keys == sorted(keys)
    assert len(set(keys)) == len(keys)


def test_config1_efficiency(cuts):
    """Plain CA on the barrel-only 50-particle events: truth efficiency >= 99 %."""
    eff = []
    for seed in range(1000, 1030):
        e = sim.generate(sim.SINGLE_MUON_LIKE, seed)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
        eff.append(truth.rates(oracle.survivors_hits(res), e.pid, e.layer)["efficiency"])
    assert np.mean(eff) >= 0.99


def test_masked_links_give_paths_of_the_kept_graph(cuts):
    """With a link mask the ntuplets are the root-to-leaf paths of the graph of kept
    links only (roots and leaves taken in that graph), and an all-true mask changes
    nothing."""
    e = sim.generate(sim.PU50, 2500, n_particles=500)
    plain = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
    same = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts,
                              link_keep=np.ones(plain["link_a"].size, bool))
    assert np.array_equal(oracle.survivors_hits(plain), oracle.survivors_hits(same))
    keep = np.random.default_rng(1).random(plain["link_a"].size) < 0.6
    res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, link_keep=keep)
    assert res["link_a"].size == keep.sum()
    G = nx.DiGraph()
    G.add_nodes_from(range(plain["cell_inner"].size))
    G.add_edges_from(zip(plain["link_a"][keep].tolist(), plain["link_b"][keep].tolist()))
    leaves = [v for v in G if G.out_degree(v) == 0]
    exp = set()
    for root in (v for v in G if G.in_degree(v) == 0 and G.out_degree(v) > 0):
        exp.update(tuple(p) for p in nx.all_simple_paths(G, root, leaves))
    got = {tuple(res["nt_cells"][t][: res["nt_n"][t] - 1].tolist()) for t in range(res["nt_n"].size)}
    assert got == exp and len(exp) > 50
