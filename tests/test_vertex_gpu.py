"""GPU parity of the primary-vertex stage (pt_find_vertices / pt_get_vertices) against
the float64 oracle (oracle/vertex.py) run on the oracle's own fitted tracks.

The ntuplets, and so the tracks and their order, are bit-exact on both sides; the
fitted z0 differ by the float32 fit error, so a cut between two consecutive tracks is
compared only where its step is farther from dz than the two tracks' z0 differences
between the sides (the groups on either side of a closer step are left out, and their
number is bounded).  Vertex z is compared within those differences plus the float32
rounding of the sum; sum of pT^2 within the fit's pT tolerance.
"""

import numpy as np
import pytest

import oracle
import sim
from oracle import vertex

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

CAP = pt.default_capacity(max_events=6, hits_per_event=65536, cells_per_event=4 << 20,
                          links_per_event=1 << 20, ntuplets_per_event=1 << 19)
DZ = vertex.DZ_DEFAULT


def _groups(track_vertex):
    out = {}
    for t, v in enumerate(track_vertex.tolist()):
        if v >= 0:
            out.setdefault(v, set()).add(t)
    return out


def _check_event(e, ev, ref, gv, goff, gtv, tr_off, gtracks, min_hits, dz):
    """One event: GPU vertices (global indices) against the oracle's."""
    hits = oracle.survivors_hits(ref)
    nh = (hits >= 0).sum(axis=1)
    fit = ref["fit"]
    z_ref = fit[:, oracle.FIT_FIELDS.index("z0")]
    pt_ref = fit[:, oracle.FIT_FIELDS.index("pt")]
    rv, rtv = vertex.find_vertices(z_ref, pt_ref, nh, min_hits=min_hits, dz=dz)
    tr = gtracks[tr_off[e]:tr_off[e + 1]]
    assert tr.shape[0] == hits.shape[0]
    z_gpu = tr["z0"].astype(np.float64)
    delta = np.abs(z_gpu - z_ref)
    # steps of the oracle's order that lie too close to dz to be decided the same way
    used = np.nonzero((nh >= min_hits) & np.isfinite(z_ref))[0]
    order = used[np.lexsort((used, z_ref[used]))]
    near = set()
    if order.size > 1:
        step = np.diff(z_ref[order])
        slack = delta[order[1:]] + delta[order[:-1]] + 1e-6
        for k in np.nonzero(np.abs(step - dz) <= slack)[0]:
            near.update((int(order[k]), int(order[k + 1])))
    assert len(near) <= max(4, int(0.02 * max(order.size, 1)))
    # groups of both sides, without those that touch an undecidable step
    v0, v1 = int(goff[e]), int(goff[e + 1])
    local = np.where(gtv[tr_off[e]:tr_off[e + 1]] >= 0, gtv[tr_off[e]:tr_off[e + 1]] - v0, -1)
    assert np.all((local == -1) | ((local >= 0) & (local < v1 - v0)))
    gg = _groups(local)
    rg = _groups(rtv)
    keep_g = {frozenset(m): v for v, m in gg.items() if not (m & near)}
    keep_r = {frozenset(m): v for v, m in rg.items() if not (m & near)}
    assert set(keep_g) == set(keep_r)
    ev_v = gv[v0:v1]
    assert np.all(ev_v["event"] == e)
    assert np.all(np.diff(ev_v["z"]) > 0)  # z order
    for members, vg in keep_g.items():
        vr = keep_r[members]
        m = np.fromiter(members, int)
        assert ev_v["n_tracks"][vg] == len(m) == rv[vr, 2]
        tol = delta[m].max() + (len(m) + 2) * 2.0 ** -23 * np.abs(z_ref[m]).mean() + 1e-6
        assert abs(float(ev_v["z"][vg]) - rv[vr, 0]) <= tol
        assert abs(float(ev_v["sum_pt2"][vg]) - rv[vr, 1]) <= 5e-4 * rv[vr, 1] + 1e-6
    return len(keep_g), len(rg)


@pytest.mark.parametrize("min_hits", [4, 3])
def test_vertices_match_oracle(cuts, min_hits):
    """A batch of vertex events of pileup 20, 90 and 200 (the last sorts more than 4096
    tracks in one block), an empty event and a two-particle event."""
    empty = sim.vertex_event(7204, 1)
    for f in ("x", "y", "z", "layer", "pid"):
        setattr(empty, f, getattr(empty, f)[:0])
    events = [sim.vertex_event(7200, 20), empty, sim.vertex_event(7201, 90),
              sim.generate(sim.SINGLE_MUON_LIKE, 1005, n_particles=2), sim.vertex_event(7202, 200)]
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_load_batch(*sim.concat(events))
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_find_ntuplets()
        ctx.pt_fit_tracks()
        nv = ctx.pt_find_vertices(min_hits=min_hits, dz=DZ)
        gv, goff, gtv = ctx.pt_get_vertices()
        _, _, tr_off = ctx.pt_get_ntuplets()
        gtracks = ctx.pt_get_tracks()
    assert nv == gv.shape[0] == goff[-1] and goff[0] == 0
    assert gtv.shape[0] == gtracks.shape[0]
    compared = total = 0
    for e, ev in enumerate(events):
        if ev.n_hits == 0:
            assert goff[e + 1] == goff[e]
            continue
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        c, t = _check_event(e, ev, ref, gv, goff, gtv, tr_off, gtracks, min_hits, DZ)
        compared += c
        total += t
    assert total > 100 and compared >= total - max(4, total // 50)


def test_vertex_errors(cuts):
    ev = sim.vertex_event(7203, 10)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_load_batch(*sim.concat([ev]))
        with pytest.raises(pt.PtError) as err:
            ctx.pt_get_vertices()
        assert err.value.status == pt.PT_ERR_INVALID
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_find_ntuplets()
        ctx.pt_fit_tracks()
        for bad in (dict(dz=0.0), dict(dz=float("nan")), dict(min_hits=2), dict(min_hits=7)):
            with pytest.raises(pt.PtError) as err:
                ctx.pt_find_vertices(**bad)
            assert err.value.status == pt.PT_ERR_INVALID
        assert ctx.pt_find_vertices() >= 1
        # a new batch invalidates the vertices of the old one
        ctx.pt_load_batch(*sim.concat([ev]))
        with pytest.raises(pt.PtError):
            ctx.pt_get_vertices()
