"""Comparison helpers for GPU-vs-oracle parity (test code; the oracle lives in oracle/)."""

from __future__ import annotations

import math

import numpy as np

# Fit tolerance: |p_gpu - p_ref| <= 1e-4 * max(|p_ref|, floor_p).  Floors (cm^-1, rad,
# cm, 1, cm) cover parameters near zero, where float32 cannot give 1e-4 relative.
FIT_REL = 1e-4
FIT_FLOORS = dict(kappa=1e-3, phi0=1.0, d0=1.0, cot_theta=1.0, z0=1.0)
# chi2: float32 residuals carry ~1e-6 cm of rounding (1e-3 of the 10 um resolution), so a
# term (eps/sigma)^2 moves by ~2e-3 |eps/sigma|; 1e-2 * max(chi2, 1) covers six hits.
CHI2_REL = 1e-2


def near_hits(ref: dict) -> set:
    """Hits taking part in a cut decision within 1e-6 relative of its threshold."""
    s = set()
    for kind, h0, h1, h2 in ref["near"].tolist():
        s.update(h for h in (h0, h1, h2) if h >= 0)
    return s


def drop_near(rows: np.ndarray, near: set) -> np.ndarray:
    if not near:
        return rows
    keep = [not (set(r[r >= 0].tolist()) & near) for r in rows]
    return rows[np.asarray(keep, bool)] if len(keep) else rows


def assert_ntuplets_equal(got: np.ndarray, exp: np.ndarray, ref: dict):
    """Cleaned ntuplets: bit-exact in canonical order.  Ntuplets sharing a hit with a
    near-threshold decision are excluded first (their number is bounded at 0.5 %); the
    full sets are then also required to agree, since both sides evaluate the cuts in
    the same float32 order."""
    near = near_hits(ref)
    g2, e2 = drop_near(got, near), drop_near(exp, near)
    assert e2.shape[0] >= exp.shape[0] - max(2, int(5e-3 * exp.shape[0]))
    assert g2.shape == e2.shape and np.array_equal(g2, e2), "ntuplets differ (near excluded)"
    assert got.shape == exp.shape and np.array_equal(got, exp), "ntuplets differ"


def cell_set(inner, outer):
    return set(zip(np.asarray(inner).tolist(), np.asarray(outer).tolist()))


def oracle_link_triples(ref: dict):
    ci, co = ref["cell_inner"], ref["cell_outer"]
    a, b = ref["link_a"], ref["link_b"]
    return dict(zip(zip(ci[a].tolist(), co[a].tolist(), co[b].tolist()),
                    ref["link_q"].view(np.uint32).tolist()))


def assert_fits_close(tracks: np.ndarray, fit: np.ndarray):
    """GPU float32 tracks vs oracle float64 fits (oracle FIT_FIELDS order)."""
    assert tracks.shape[0] == fit.shape[0]
    if fit.shape[0] == 0:
        return
    cols = dict(kappa=0, phi0=1, d0=2, cot_theta=3, z0=4)
    for name, c in cols.items():
        g = tracks[name].astype(np.float64)
        r = fit[:, c]
        if name == "phi0":
            d = np.abs(np.remainder(g - r + math.pi, 2 * math.pi) - math.pi)
        else:
            d = np.abs(g - r)
        tol = FIT_REL * np.maximum(np.abs(r), FIT_FLOORS[name])
        bad = np.flatnonzero(d > tol)
        assert bad.size == 0, (f"{name}: {bad.size} of {r.size} outside tolerance, worst "
                               f"{np.max(d / tol):.3g} x tol at ref {r[bad[0]]}")
    assert np.array_equal(tracks["charge"].astype(np.float64), fit[:, 8])
    for name, c in (("chi2_circle", 6), ("chi2_line", 7)):
        g = tracks[name].astype(np.float64)
        r = fit[:, c]
        assert np.all(np.abs(g - r) <= CHI2_REL * np.maximum(np.abs(r), 1.0)), name
