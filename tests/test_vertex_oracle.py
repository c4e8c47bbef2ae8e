"""Pins of the vertexing oracle (oracle/vertex.py) against a hand-worked case, the
single-linkage definition by brute force, and generator truth on noiseless events."""

import numpy as np
import pytest

import oracle
import sim
from oracle import vertex
from sim import truth


def test_hand_worked_groups():
    # steps of exactly dz do not cut; a 3-hit track, a NaN z0 and a lone track are not used
    z0 = np.array([4.25, 0.0, 10.0, 0.375, 4.0, 0.125, 0.2, np.nan])
    pt = np.array([1.0, 1.0, 5.0, 3.0, 1.0, 2.0, 7.0, 1.0])
    nh = np.array([4, 4, 5, 6, 4, 4, 3, 4])
    v, tv = vertex.find_vertices(z0, pt, nh, min_hits=4, dz=0.25)
    assert v.shape == (2, 3)
    np.testing.assert_allclose(v[0], [0.5 / 3.0, 1.0 + 4.0 + 9.0, 3.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(v[1], [8.25 / 2.0, 2.0, 2.0], rtol=0, atol=1e-15)
    assert tv.tolist() == [1, 0, -1, 0, 1, 0, -1, -1]


def test_equal_z0_and_empty_inputs():
    v, tv = vertex.find_vertices([1.0, 1.0], [1.0, 2.0], [4, 4], dz=0.0)
    assert v.shape == (1, 3) and v[0, 2] == 2 and tv.tolist() == [0, 0]
    v, tv = vertex.find_vertices([], [], [], dz=0.02)
    assert v.shape == (0, 3) and tv.size == 0
    v, tv = vertex.find_vertices([0.0, 1.0], [1.0, 1.0], [4, 4], dz=0.5)
    assert v.shape == (0, 3) and tv.tolist() == [-1, -1]


@pytest.mark.parametrize("seed", range(20))
def test_sort_and_cut_equals_single_linkage(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    z0 = np.round(rng.normal(0.0, 0.2, n), 3)  # ties and steps at exactly dz occur
    dz = 0.02
    v, tv = vertex.find_vertices(z0, np.ones(n), np.full(n, 4), dz=dz)
    groups = [g for g in vertex.single_linkage_groups(z0, dz) if len(g) >= 2]
    assert v.shape[0] == len(groups)
    for k, g in enumerate(groups):
        assert sorted(np.nonzero(tv == k)[0].tolist()) == g
        assert v[k, 0] == pytest.approx(z0[g].mean(), abs=1e-12)
        assert v[k, 2] == len(g)
    assert np.all(np.diff(v[:, 0]) > dz)


def test_noiseless_vertices_are_found(cuts):
    """Noiseless hits: a quadruplet's fitted z0 is its vertex's z, so every generated
    vertex well apart from the others with at least two fully matched quadruplets gives
    one vertex at its z that holds all of them."""
    found = 0
    for seed in (7100, 7101):
        ev = sim.vertex_event(seed, 12, noise_frac=0.0, smear=False)
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        hits = oracle.survivors_hits(ref)
        fit = ref["fit"]
        nh = (hits >= 0).sum(axis=1)
        z0 = fit[:, oracle.FIT_FIELDS.index("z0")]
        pt = fit[:, oracle.FIT_FIELDS.index("pt")]
        v, tv = vertex.find_vertices(z0, pt, nh)
        part = truth.match_fast(hits, ev.pid)
        vz = ev.particles["vz"]
        tvert = np.where(part >= 0, ev.particles["vertex"][np.maximum(part, 0)], -1)
        for k in range(vz.size):
            if np.min(np.abs(np.delete(vz, k) - vz[k])) < 10 * vertex.DZ_DEFAULT:
                continue
            mine = np.nonzero((tvert == k) & (nh >= 4))[0]
            if mine.size < 2:
                continue
            near = np.nonzero(np.abs(v[:, 0] - vz[k]) < 1e-3)[0]
            assert near.size == 1, (seed, k, near)
            assert np.all(tv[mine] == near[0])
            assert abs(np.median(z0[mine]) - vz[k]) < 1e-6
            found += 1
    assert found >= 10
