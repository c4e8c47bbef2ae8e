"""The oracle's fishbone step (aligned active cells sharing an outer hit), pinned by
geometry: hand-made vectors for the comparison, straight tracks with an overlap hit or
skip-layer pairs for the chain, invariance under the input order, and the generator's
overlapping sensors."""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import sim

THRESHOLD = math.acos(math.sqrt(0.99999))  # 3.162 mrad between the two cell directions


def _rot(v, ang):
    """v turned by ang in its (x, y) plane."""
    c, s = math.cos(ang), math.sin(ang)
    return (c * v[0] - s * v[1], s * v[0] + c * v[1], v[2])


def test_collinear_same_layer_shorter_cell_loses():
    h = (10.0, 0.0, 3.0)
    near, far = (7.0, 0.0, 2.1), (6.0, 0.0, 1.8)  # both on the line from the origin
    assert oracle.fishbone_loses(h, near, 1, 0, far, 1, 1)
    assert not oracle.fishbone_loses(h, far, 1, 1, near, 1, 0)


def test_collinear_different_layers_longer_cell_loses():
    h = (10.0, 0.0, 3.0)
    near, far = (7.0, 0.0, 2.1), (3.0, 0.0, 0.9)
    assert oracle.fishbone_loses(h, far, 0, 5, near, 1, 9)
    assert not oracle.fishbone_loses(h, near, 1, 9, far, 0, 5)


@pytest.mark.parametrize("ang,aligned", [(0.9 * THRESHOLD, True), (1.1 * THRESHOLD, False)])
def test_alignment_threshold(ang, aligned):
    """Directions 0.9 and 1.1 times the threshold angle apart (in the transverse plane)."""
    h = (10.0, 0.0, 0.0)
    d1 = (-4.0, 0.0, 0.0)
    d2 = _rot((-3.0, 0.0, 0.0), ang)
    i = tuple(a + b for a, b in zip(h, d1))
    j = tuple(a + b for a, b in zip(h, d2))
    assert oracle.fishbone_loses(h, j, 1, 0, i, 1, 1) is aligned  # j: the shorter cell


def test_opposite_directions_never_align():
    h = (10.0, 0.0, 0.0)
    assert not oracle.fishbone_loses(h, (7.0, 0.0, 0.0), 1, 0, (13.0, 0.0, 0.0), 1, 1)
    assert not oracle.fishbone_loses(h, (13.0, 0.0, 0.0), 1, 1, (7.0, 0.0, 0.0), 1, 0)


def test_equal_lengths_larger_index_loses():
    h = (10.0, 0.0, 0.0)
    i, j = (7.0, 0.0, 0.0), (7.0, 0.0, 0.0)
    assert oracle.fishbone_loses(h, i, 0, 8, j, 1, 3)
    assert not oracle.fishbone_loses(h, j, 1, 3, i, 0, 8)


@pytest.mark.parametrize("layer,gap,compared", [(1, 0.05, False), (1, 0.2, True),
                                                (5, 0.05, False), (5, 0.2, True)])
def test_same_layer_needs_two_sensors(layer, gap, compared):
    """On one layer only inner hits on different sensors are compared: radii (barrel)
    or |z| (disk) more than 0.1 cm apart.  Both cells lie on one line from the outer hit."""
    if layer < 4:   # barrel: the line from the origin, hits at r and r + gap
        h, i, j = (10.0, 0.0, 4.0), (6.8, 0.0, 2.72), (6.8 + gap, 0.0, 0.4 * (6.8 + gap))
    else:           # disk: a steep line, hits at z and z + gap
        h, i, j = (8.0, 0.0, 52.0), (6.0, 0.0, 39.0), (6.0 + gap / 6.5, 0.0, 39.0 + gap)
    assert oracle.fishbone_loses(h, j, layer, 1, i, layer, 0) is compared  # j: the shorter
    assert not oracle.fishbone_loses(h, i, layer, 0, j, layer, 1)


def _line(radii, layers, phi=0.3, cot=0.4):
    r = np.asarray(radii, np.float64)
    x, y, z = r * math.cos(phi), r * math.sin(phi), r * cot
    return (x.astype(np.float32), y.astype(np.float32), z.astype(np.float32),
            np.asarray(layers, np.uint8))


def _candidates(res):
    return sorted(tuple(int(v) for v in row if v >= 0) for row in res["nt_hits"])


def _links(res):
    ci, co = res["cell_inner"], res["cell_outer"]
    return sorted(zip(ci[res["link_a"]].tolist(), co[res["link_a"]].tolist(),
                      co[res["link_b"]].tolist()))


def test_overlap_hit_cell_removed(cuts):
    """A straight track with a second hit on layer 1 (overlapping sensor, 0.5 cm further
    out): the cells (1, 2) and (1', 2) are aligned at hit 2 and the shorter (1', 2) goes,
    with both links through hit 1'."""
    x, y, z, layer = _line([2.9, 6.8, 7.3, 10.9, 16.0], [0, 1, 1, 2, 3])
    off = oracle.reconstruct(x, y, z, layer, cuts)
    on = oracle.reconstruct(x, y, z, layer, cuts, fishbone=True)
    assert _candidates(off) == [(0, 1, 3, 4), (0, 2, 3, 4)]
    assert _candidates(on) == [(0, 1, 3, 4)]
    assert set(_links(off)) - set(_links(on)) == {(0, 2, 3), (2, 3, 4)}
    # the cells themselves stay (the step removes links, not doublets)
    assert off["cell_inner"].size == on["cell_inner"].size


def test_skip_layer_cell_removed(cuts):
    """A straight track through layers 0..3 with the skip-layer pairs: at hit 2 the cells
    (1, 2) and (0, 2) are aligned on different layers and the longer (0, 2) goes; at hit
    3 the cells have no outgoing link and are not compared."""
    x, y, z, layer = _line([2.9, 6.8, 10.9, 16.0], [0, 1, 2, 3])
    pairs = oracle.DEFAULT_PAIRS + oracle.gap_pairs()
    off = oracle.reconstruct(x, y, z, layer, cuts, pairs=pairs)
    on = oracle.reconstruct(x, y, z, layer, cuts, pairs=pairs, fishbone=True)
    assert (0, 2, 3) in _links(off)
    assert _candidates(off) == [(0, 1, 2, 3), (0, 1, 3), (0, 2, 3)]
    assert _candidates(on) == [(0, 1, 2, 3), (0, 1, 3)]
    assert not [lk for lk in _links(on) if lk[:2] == (0, 2)]


def test_off_leaves_the_chain_unchanged(cuts):
    ev = sim.generate(sim.PU50, 4100)
    a = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    b = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, fishbone=False)
    for k in ("cell_inner", "link_a", "link_b", "nt_hits", "survivors", "fit"):
        assert np.array_equal(a[k], b[k])


def test_independent_of_input_order(cuts):
    """Overlap event: the removal keeps the same tracks whatever the order of the hits
    (each cell decides from the links before the removal)."""
    cfg = dataclasses.replace(sim.PU50, n_particles=600, overlap=0.3)
    ev = sim.generate(cfg, 4101)
    on = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, fishbone=True)
    off = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    assert len(_links(on)) < len(_links(off))  # the step acts on this event
    perm = np.random.default_rng(5).permutation(ev.n_hits)
    on_p = oracle.reconstruct(ev.x[perm], ev.y[perm], ev.z[perm], ev.layer[perm], cuts,
                              fishbone=True)
    back = lambda rows: sorted(tuple(sorted(perm[v] for v in r if v >= 0)) for r in rows)
    fwd = lambda rows: sorted(tuple(sorted(v for v in r if v >= 0)) for r in rows)
    assert back(oracle.survivors_hits(on_p)) == fwd(oracle.survivors_hits(on))
    assert back(on_p["nt_hits"]) == fwd(on["nt_hits"])


def test_overlapping_sensors_in_the_generator():
    cfg = dataclasses.replace(sim.SINGLE_MUON_LIKE, overlap=1.0, smear=False, noise_frac=0.0)
    ev = sim.generate(cfg, 4102)
    base = sim.generate(dataclasses.replace(cfg, overlap=0.0), 4102)
    r = np.hypot(ev.x64, ev.y64)
    for L, rl in enumerate(sim.events.BARREL_R):
        m = ev.layer == L
        radii = np.unique(np.round(r[m], 6))
        assert set(radii) <= {round(rl, 6), round(rl + sim.events.OVERLAP_DR, 6)}
    # every particle gains at most one hit per layer, on the same layer
    for p in np.unique(base.pid):
        a = np.bincount(base.layer[base.pid == p], minlength=10)
        b = np.bincount(ev.layer[ev.pid == p], minlength=10)
        assert np.all((b == a) | (b == a + 1))
    assert ev.n_hits > 1.5 * base.n_hits
