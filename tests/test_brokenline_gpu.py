"""GPU parity of the broken-line refit (pt_refit_broken_line) against the float64
oracle (oracle/brokenline.py) run on the oracle's own ntuplets and fits.

The ntuplets are bit-exact on both sides, so the refits are compared track by track:
parameters within 1e-4 relative (the circle fit's floors), chi2 within 1e-2 relative.
The GPU's reference is its float32 circle fit and the oracle's its float64 one; a
broken-line solution depends on its reference only at second order (the pins show
1e-7 from a 1e-3 offset), and the GPU computes everything after its float32 loads in
float64, so the comparison is limited by the float32 outputs.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import sim
from oracle import brokenline as bl
from parity import CHI2_REL, FIT_FLOORS, assert_fits_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

CAP = pt.default_capacity(max_events=6, hits_per_event=65536, cells_per_event=4 << 20,
                          links_per_event=1 << 20, ntuplets_per_event=1 << 19)
MAT = dict(x0_barrel=0.02, x0_disk=0.02)


def _events():
    pu50 = dataclasses.replace(sim.PU50, **MAT)
    pu200 = dataclasses.replace(sim.PU200, **MAT)
    return [sim.generate(pu50, 2100), sim.generate(sim.PU50, 2101),
            sim.generate(pu200, 3150)]


def _chain(ctx, events):
    ctx.pt_load_batch(*sim.concat(events))
    ctx.pt_build_doublets()
    ctx.pt_connect_cells()
    ctx.pt_find_ntuplets()
    ctx.pt_fit_tracks()


def _oracle_refits(ev, cuts, x0b, x0d):
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    hits = oracle.survivors_hits(ref)
    nh = (hits >= 0).sum(axis=1)
    x, y, z = (a.astype(np.float64) for a in (ev.x, ev.y, ev.z))
    return ref, hits, nh, bl.refit_tracks(x, y, z, ev.layer, hits, nh, ref["fit"], x0b, x0d)


def _assert_chi2_close(tracks, fit):
    for name, c in (("chi2_circle", 6), ("chi2_line", 7)):
        g = tracks[name].astype(np.float64)
        r = fit[:, c]
        assert np.all(np.abs(g - r) <= CHI2_REL * np.maximum(np.abs(r), 1.0)), name


@pytest.mark.parametrize("x0b,x0d", [(0.02, 0.02), (0.015, 0.035)])
def test_refit_matches_oracle(cuts, x0b, x0d):
    """PU50 and PU200 events whose particles scatter in 2 % X0 per layer, and a PU50
    event without material (the refit assumes material all the same)."""
    events = _events()
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        _chain(ctx, events)
        circle = ctx.pt_get_tracks()
        n = ctx.pt_refit_broken_line(x0b, x0d)
        tracks = ctx.pt_get_tracks()
        _, _, off = ctx.pt_get_ntuplets()
    assert n == tracks.shape[0] == circle.shape[0]
    assert np.array_equal(tracks["nhits"], circle["nhits"])
    matched_bl, matched_circle, ndf = 0.0, 0.0, 0
    for e, ev in enumerate(events):
        ref, hits, nh, exp = _oracle_refits(ev, cuts, x0b, x0d)
        sl = slice(off[e], off[e + 1])
        assert off[e + 1] - off[e] == exp.shape[0] > 500
        assert_fits_close(tracks[sl], exp)
        _assert_chi2_close(tracks[sl], exp)
        if e == 1:
            continue
        # what the refit is for: on tracks of one particle its transverse chi2 per
        # degree of freedom is near 1, the scattering-blind circle fit's is not
        pid = np.where(hits >= 0, ev.pid[np.maximum(hits, 0)], -2)
        one = np.array([len(set(r[:k].tolist())) == 1 and r[0] >= 0 for r, k in zip(pid, nh)])
        m = one & (nh >= 4)
        matched_bl += float(tracks[sl]["chi2_circle"][m].sum())
        matched_circle += float(circle[sl]["chi2_circle"][m].sum())
        ndf += int((nh[m] - 3).sum())
    assert ndf > 1000
    assert 0.7 < matched_bl / ndf < 1.5
    assert matched_circle / ndf > 2.0 * matched_bl / ndf


def test_refit_of_a_refit_is_stable(cuts):
    """A second refit takes the first as its reference and lands on the same tracks
    within the passes' stopping precision (a pass that moves the curvature by at most
    1e-3 relative ends them; the slope weights follow the reference, so z0 and
    cot(theta) settle to the same order): 1e-3 relative with the circle fit's floors."""
    events = _events()[:1]
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        _chain(ctx, events)
        ctx.pt_refit_broken_line(**MAT)
        a = ctx.pt_get_tracks()
        ctx.pt_refit_broken_line(**MAT)
        b = ctx.pt_get_tracks()
    assert np.array_equal(a["charge"], b["charge"])
    for name, floor in FIT_FLOORS.items():
        r = a[name].astype(np.float64)
        d = np.abs(b[name].astype(np.float64) - r)
        if name == "phi0":
            d = np.abs(np.remainder(d + np.pi, 2 * np.pi) - np.pi)
        assert np.all(d <= 1e-3 * np.maximum(np.abs(r), floor)), name


def test_refit_errors(cuts):
    ev = sim.generate(sim.PU50, 2102)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        with pytest.raises(pt.PtError) as err:  # nothing loaded
            ctx.pt_refit_broken_line()
        assert err.value.status == pt.PT_ERR_INVALID
        ctx.pt_load_batch(*sim.concat([ev]))
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_find_ntuplets()
        with pytest.raises(pt.PtError) as err:  # not fitted yet
            ctx.pt_refit_broken_line()
        assert err.value.status == pt.PT_ERR_INVALID
        ctx.pt_fit_tracks()
        for bad in ((0.0, 0.02), (0.02, -1.0), (1.5, 0.02), (float("nan"), 0.02)):
            with pytest.raises(pt.PtError) as err:
                ctx.pt_refit_broken_line(*bad)
            assert err.value.status == pt.PT_ERR_INVALID
        assert ctx.pt_refit_broken_line() > 100
