"""Pins of the oracle's skip-layer (gap) doublet mode: the pair table it derives, the
default table left untouched, cells against the geometric definition on every pair of
the extended table, ntuplets as the maximal chains of its link graph, and what the
mode gains on events with inefficient sensors."""

import dataclasses

import networkx as nx
import numpy as np
import pytest

import oracle
import sim
from sim import truth
from test_oracle_pins import _clear, _f64, _tiny_event

FULL = oracle.DEFAULT_PAIRS + oracle.gap_pairs()


def test_gap_pairs_by_hand():
    """Two steps on the pair graph that are not already a pair: barrel 0-2 and 1-3,
    barrel to the second disk of either side, the first to the third disk."""
    assert oracle.gap_pairs() == ((0, 2), (0, 5), (0, 8), (1, 3), (1, 5), (1, 8), (2, 5),
                                  (2, 8), (4, 6), (7, 9))
    assert oracle.DEFAULT_PAIRS == truth.LAYER_PAIRS


def test_default_table_gives_the_default_chain(cuts):
    e = sim.generate(sim.PU50, 2300, n_particles=800)
    a = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts)
    b = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, pairs=oracle.DEFAULT_PAIRS)
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), k
        else:
            assert a[k] == b[k], k


def test_invalid_tables_are_refused(cuts):
    e = sim.generate(sim.SINGLE_MUON_LIKE, 1000)
    for bad in ([(0, 0)], [(0, 10)], [(-1, 2)], [], [(0, 1)] * 65, [(0, 1), (0, 1)],
                [(0, 1), (1, 2), (0, 1)]):
        with pytest.raises(ValueError):
            oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, pairs=bad)


def test_gap_doublets_match_geometric_definition(cuts):
    """Cells of the extended table: every hit pair on one of its 23 layer pairs that is
    outward, within 90 degrees in azimuth, on a circle through the beam spot of
    curvature <= kmax, with |z0| <= z0max and |dz/dr| <= cotmax."""
    n_checked = n_skipped = 0
    for seed in range(8):
        e = _tiny_event(300 + seed)
        res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, pairs=FULL)
        got = set(zip(res["cell_inner"].tolist(), res["cell_outer"].tolist()))
        x, y, z, r = _f64(e)
        phi = np.arctan2(y, x)
        exp, amb = set(), set()
        gap_cells = 0
        for li, lo in FULL:
            I = np.flatnonzero(e.layer == li)
            O = np.flatnonzero(e.layer == lo)
            if I.size == 0 or O.size == 0:
                continue
            i, o = np.meshgrid(I, O, indexing="ij")
            i, o = i.ravel(), o.ravel()
            dphi = np.angle(np.exp(1j * (phi[o] - phi[i])))
            kappa = 2.0 * np.abs(np.sin(dphi)) / np.hypot(x[o] - x[i], y[o] - y[i])
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
                    gap_cells += (li, lo) not in oracle.DEFAULT_PAIRS
            n_checked += i.size
        n_skipped += len(amb)
        assert gap_cells > 10
        assert (got - amb) == exp, f"seed {seed}"
    assert n_skipped < 1e-3 * n_checked


def test_gap_ntuplets_are_the_maximal_chains(cuts):
    """Ntuplets of the extended table are exactly the root-to-leaf paths (>= 2 cells) of
    its link graph, and every step of their layer sequence is a pair of the table."""
    allowed = set(FULL)
    e = sim.generate(dataclasses.replace(sim.PU50, hit_eff=0.9), 2310, n_particles=500)
    res = oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, pairs=FULL)
    G = nx.DiGraph()
    G.add_nodes_from(range(res["cell_inner"].size))
    G.add_edges_from(zip(res["link_a"].tolist(), res["link_b"].tolist()))
    leaves = [v for v in G if G.out_degree(v) == 0]
    exp = set()
    for root in (v for v in G if G.in_degree(v) == 0 and G.out_degree(v) > 0):
        exp.update(tuple(p) for p in nx.all_simple_paths(G, root, leaves))
    got = set()
    n_gap = 0
    for t in range(res["nt_n"].size):
        n = int(res["nt_n"][t])
        cells = res["nt_cells"][t][: n - 1].tolist()
        hits = res["nt_hits"][t][:n].tolist()
        lay = e.layer[hits].tolist()
        assert all((u, v) in allowed for u, v in zip(lay[:-1], lay[1:]))
        n_gap += any((u, v) not in oracle.DEFAULT_PAIRS for u, v in zip(lay[:-1], lay[1:]))
        got.add(tuple(cells))
    assert got == exp and len(exp) > 100 and n_gap > 20


def test_gap_pairs_recover_tracks_with_missing_hits(cuts):
    """With 10 % of the crossings lost, chains that step over a missing surface are
    found: efficiency (particles with a >= 3-hit chain on the extended table) rises by
    more than 8 points over the default table (73 % -> 85 % on this event), and with
    every crossing present the mode loses nothing."""
    for eff, gain in ((0.9, 0.08), (1.0, 0.0)):
        e = sim.generate(dataclasses.replace(sim.PU50, hit_eff=eff), 2200)
        plain = oracle.survivors_hits(oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts))
        gap = oracle.survivors_hits(oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts, pairs=FULL))
        rp = truth.rates_fast(plain, e.pid, e.layer, pairs=FULL)
        rg = truth.rates_fast(gap, e.pid, e.layer, pairs=FULL)
        assert rg["efficiency"] >= rp["efficiency"] + gain, (eff, rp, rg)


def test_inefficiency_drops_crossings_independently():
    """hit_eff keeps each crossing with that probability; 1 leaves events unchanged."""
    a = sim.generate(sim.PU50, 2000)
    b = sim.generate(dataclasses.replace(sim.PU50, hit_eff=1.0), 2000)
    assert np.array_equal(a.x64, b.x64)
    c = sim.generate(dataclasses.replace(sim.PU50, hit_eff=0.8, noise_frac=0.0), 2001)
    d = sim.generate(dataclasses.replace(sim.PU50, noise_frac=0.0), 2001)
    assert abs(c.n_hits / d.n_hits - 0.8) < 0.02
