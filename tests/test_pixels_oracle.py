"""Pins of the raw-data oracle (oracle/pixels.py): a hand-worked module, the
8-neighbourhood definition by brute force, and the true positions of isolated hits."""

import math
import os

import numpy as np
import pytest

import sim
from oracle import pixels
from sim import pixels as simpix

PARAMS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2501_05520_gb300", "params", "pixels_v1.json")


@pytest.fixture(scope="module")
def table():
    return pixels.modules(PARAMS)


def _pack(m, r, c, a):
    return (m << 40) | (r << 28) | (c << 16) | a


def test_module_table_by_hand(table):
    assert table.shape == ((12 + 28 + 44 + 64) * 8 + 6 * 48 * 2, 9)
    # first module: layer 0, sector 0, segment 0; 2 pi 2.9 / 12 = 1.518 cm -> 152 columns,
    # 6.75 cm / 0.015 cm -> 450 rows
    assert table[0].tolist() == pytest.approx([0, 0, 2.9, -math.pi, 2 * math.pi / 12 / 152, -27.0,
                                               0.015, 152, 450])
    # first -z disk module (layer 7): ring 0 of (16 - 4.5) / 2 cm centred at 7.375 cm,
    # 48 sectors -> ceil(7.375 x 2 pi / 48 / 0.01) = 97 columns, 5.75 / 0.015 -> 384 rows
    k = (12 + 28 + 44 + 64) * 8 + 3 * 96
    assert table[k].tolist() == pytest.approx([7, 1, -29.1, -math.pi, 2 * math.pi / 48 / 97, 4.5,
                                               0.015, 97, 384])
    # the generator's own table (written separately) agrees
    mt = simpix.module_table()
    for i, f in enumerate(pixels.MODULE_FIELDS):
        np.testing.assert_allclose(mt[f], table[:, i], rtol=0, atol=1e-12)


def test_hand_worked_module(table):
    m = 100
    pix = [(5, 5, 10), (5, 6, 30), (11, 11, 7), (10, 10, 9), (20, 20, 50), (30, 30, 4),
           (30, 32, 6)]
    words = np.asarray([_pack(m, r, c, a) for r, c, a in pix], np.uint64)
    x, y, z, layer, members = pixels.reconstruct(words, table)
    assert [g.tolist() for g in members] == [[0, 1], [2, 3], [4], [5], [6]]
    col_c = [(10 * 5.5 + 30 * 6.5) / 40, (7 * 11.5 + 9 * 10.5) / 16, 20.5, 30.5, 32.5]
    row_c = [5.5, (7 * 11.5 + 9 * 10.5) / 16, 20.5, 30.5, 30.5]
    mod = table[m]
    for h in range(5):
        phi = mod[3] + col_c[h] * mod[4]
        assert x[h] == pytest.approx(mod[2] * math.cos(phi), abs=1e-12)
        assert y[h] == pytest.approx(mod[2] * math.sin(phi), abs=1e-12)
        assert z[h] == pytest.approx(mod[5] + row_c[h] * mod[6], abs=1e-12)
    assert np.all(layer == mod[0])


@pytest.mark.parametrize("seed", range(15))
def test_components_equal_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 80))
    cells = {(int(r), int(c)) for r, c in rng.integers(0, 12, (n, 2))}
    rows = np.asarray([p[0] for p in sorted(cells)])
    cols = np.asarray([p[1] for p in sorted(cells)])
    lab = pixels._components(rows, cols)
    got = {}
    for i, root in enumerate(lab):
        got.setdefault(root, []).append(i)
    assert sorted(sorted(g) for g in got.values()) == pixels.components_brute_force(rows, cols)
    assert all(root == min(g) for root, g in got.items())


def test_isolated_hits_come_back(table):
    """Noiseless single particles: every hit is alone on its module, so its cluster's
    centroid returns the true crossing up to the adc rounding (a few micrometres)."""
    checked = 0
    for k, (pt, eta) in enumerate([(1.0, 0.3), (3.0, -1.2), (0.7, 2.0), (5.0, -2.2)]):
        ev = sim.single_helix(50 + k, pt, eta, 0.4 + k, 1.0 if k % 2 else -1.0, 0.5 * k,
                              barrel_only=False)
        words, owner, _ = simpix.digitize(ev)
        x, y, z, layer, members = pixels.reconstruct(words, table)
        assert x.size == ev.n_hits
        for h in range(x.size):
            src = set(owner[members[h]].tolist())
            assert len(src) == 1
            t = src.pop()
            assert layer[h] == ev.layer[t]
            d = math.hypot(x[h] - ev.xt[t], y[h] - ev.yt[t])
            assert d < 5e-4 and abs(z[h] - ev.zt[t]) < 5e-4, (h, d, z[h] - ev.zt[t])
            checked += 1
    assert checked >= 15
