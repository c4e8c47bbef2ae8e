"""GPU parity: the CUDA chain against the CPU oracle, element by element.

Cells, links (with their float32 quality), ntuplet candidates and cleaned ntuplets
must be bit-exact; fitted parameters within 1e-4 relative of the float64 oracle fit
(floors in parity.py).  Every call goes through the C ABI via the thin binding.
"""

import numpy as np
import pytest

import oracle
import sim
from parity import (assert_fits_close, assert_ntuplets_equal, cell_set, oracle_link_triples)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

SMALL_CAP = pt.default_capacity(max_events=8, hits_per_event=4096, cells_per_event=1 << 16,
                                links_per_event=1 << 15, ntuplets_per_event=1 << 14)
PU_CAP = pt.default_capacity(max_events=2, hits_per_event=65536, cells_per_event=4 << 20,
                             links_per_event=1 << 20, ntuplets_per_event=1 << 19)


@pytest.fixture(scope="module")
def small_ctx(cuts):
    with pt.Context(cuts=cuts, capacity=SMALL_CAP) as c:
        yield c


@pytest.fixture(scope="module")
def pu_ctx(cuts):
    with pt.Context(cuts=cuts, capacity=PU_CAP) as c:
        yield c


def run_stages(ctx, events):
    off, x, y, z, layer = sim.concat(events)
    ctx.pt_load_batch(off, x, y, z, layer)
    out = dict(n_cells=ctx.pt_build_doublets(), n_links=ctx.pt_connect_cells(),
               n_nt=ctx.pt_find_ntuplets(), n_tracks=ctx.pt_fit_tracks())
    out["cells"] = ctx.pt_get_cells()
    out["links"] = ctx.pt_get_links()
    out["cand"] = ctx.pt_get_candidates()
    out["nt"] = ctx.pt_get_ntuplets()
    out["tracks"] = ctx.pt_get_tracks()
    return out


def check_event(out, e, ev, ref, edge_cases=False):
    """edge_cases: the event was built on the cuts' edges, so the bound on ntuplets near a
    threshold does not apply; the full sets must still be equal."""
    ci, co, ce = out["cells"]
    m = ce == e
    assert cell_set(ci[m], co[m]) == cell_set(ref["cell_inner"], ref["cell_outer"])
    h0, h1, h2, q, le = out["links"]
    m = le == e
    got = dict(zip(zip(h0[m].tolist(), h1[m].tolist(), h2[m].tolist()),
                   q[m].view(np.uint32).tolist()))
    assert got == oracle_link_triples(ref)
    hits, nh, cq, cev = out["cand"]
    m = cev == e
    got_c = {tuple(r): v for r, v in zip(hits[m].tolist(), cq[m].view(np.uint32).tolist())}
    exp_c = {tuple(r): v for r, v in zip(ref["nt_hits"].tolist(),
                                         ref["nt_q"].view(np.uint32).tolist())}
    assert got_c == exp_c
    assert int(m.sum()) == ref["nt_n"].size  # no duplicate candidates
    nth, ntn, evoff = out["nt"]
    sl = slice(evoff[e], evoff[e + 1])
    if edge_cases:
        assert np.array_equal(nth[sl], oracle.survivors_hits(ref))
    else:
        assert_ntuplets_equal(nth[sl], oracle.survivors_hits(ref), ref)
    assert np.array_equal(ntn[sl], ref["nt_n"][ref["survivors"]].astype(np.uint8))
    assert_fits_close(out["tracks"][sl], ref["fit"])


def test_config1_batch_matches_oracle(small_ctx, cuts):
    events = [sim.generate(sim.SINGLE_MUON_LIKE, 1000 + i) for i in range(8)]
    out = run_stages(small_ctx, events)
    for e, ev in enumerate(events):
        check_event(out, e, ev, oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts))


def test_pu50_event_matches_oracle(cuts_low_pt):
    with pt.Context(cuts=cuts_low_pt, capacity=PU_CAP) as ctx:
        ev = sim.generate(sim.PU50, 2000)
        out = run_stages(ctx, [ev])
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts_low_pt)
        assert out["n_cells"] == ref["cell_inner"].size
        check_event(out, 0, ev, ref)


def test_pu200_event_matches_oracle(pu_ctx, cuts):
    ev = sim.generate(sim.PU200, 3000)
    out = run_stages(pu_ctx, [ev])
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    assert out["n_cells"] > 1_000_000
    check_event(out, 0, ev, ref)


def test_graph_path_equals_stage_path(pu_ctx, cuts):
    events = [sim.generate(sim.PU50, 2010), sim.generate(sim.PU50, 2011, n_particles=700)]
    out = run_stages(pu_ctx, events)
    off, x, y, z, layer = sim.concat(events)
    hits, nh, tracks, evoff = pu_ctx.pt_reconstruct_batch(off, x, y, z, layer)
    assert np.array_equal(hits, out["nt"][0])
    assert np.array_equal(evoff, out["nt"][2])
    assert tracks.tobytes() == out["tracks"].tobytes()


def test_uneven_batch_with_empty_and_degenerate_events(small_ctx, cuts):
    g = sim.GenConfig(60, "inv_pt_uniform", 2.5, False, 0.3)
    full = sim.generate(g, 77)
    one_layer = sim.generate(g, 78)
    keep = one_layer.layer == 1
    for f in ("x", "y", "z", "layer", "pid"):
        setattr(one_layer, f, getattr(one_layer, f)[keep])
    empty = sim.generate(g, 79)
    for f in ("x", "y", "z", "layer", "pid"):
        setattr(empty, f, getattr(empty, f)[:0])
    events = [empty, full, one_layer, sim.generate(g, 80, n_particles=7), empty,
              sim.generate(sim.SINGLE_MUON_LIKE, 1005)]
    out = run_stages(small_ctx, events)
    evoff = out["nt"][2]
    assert evoff.size == len(events) + 1
    for e, ev in enumerate(events):
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        check_event(out, e, ev, ref)
    assert evoff[1] == evoff[0] == 0 and evoff[5] == evoff[4]


@pytest.mark.parametrize("bins", [16, 4096])
def test_phi_binning_is_only_an_acceleration(cuts, bins):
    cap = dict(PU_CAP, phi_bins=bins)
    ev = sim.generate(sim.PU50, 2020, n_particles=800)
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        out = run_stages(ctx, [ev])
    check_event(out, 0, ev, oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts))


def test_repeat_is_deterministic(pu_ctx):
    ev = sim.generate(sim.PU50, 2030)
    a = pu_ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
    a = [np.copy(v) for v in a]
    for _ in range(2):
        b = pu_ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
        assert all(np.array_equal(u, v) for u, v in zip(a[:2] + a[3:], b[:2] + b[3:]))
        assert a[2].tobytes() == b[2].tobytes()


def test_device_inputs(pu_ctx, cuts):
    ev = sim.generate(sim.PU50, 2040, n_particles=500)
    d = [torch.from_numpy(v).cuda() for v in (ev.x, ev.y, ev.z, ev.layer)]
    hits, nh, tracks, evoff = pu_ctx.pt_reconstruct_batch([0, ev.n_hits], *d)
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    assert_ntuplets_equal(hits, oracle.survivors_hits(ref), ref)
    out = dict(hits=torch.empty((4096, 6), dtype=torch.int32, device="cuda"),
               nhits=torch.empty(4096, dtype=torch.uint8, device="cuda"),
               tracks=torch.empty((4096, 36), dtype=torch.uint8, device="cuda"),
               event_offsets=torch.empty(2, dtype=torch.int64, device="cuda"))
    h2, n2, t2, o2 = pu_ctx.pt_reconstruct_batch([0, ev.n_hits], *d, out=out)
    assert np.array_equal(h2.cpu().numpy(), hits)
    assert t2.cpu().numpy().tobytes() == tracks.tobytes()


def test_capacity_and_input_errors(cuts):
    ev = sim.generate(sim.PU50, 2050, n_particles=400)
    cap = pt.default_capacity(max_events=1, hits_per_event=8192, cells_per_event=1000,
                              links_per_event=1000, ntuplets_per_event=1000)
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_build_doublets()
        assert ei.value.status == pt.PT_ERR_CAPACITY and "max_cells" in str(ei.value)
        big = sim.generate(sim.PU50, 2051)
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_load_hits(big.x, big.y, big.z, big.layer)
        assert ei.value.status == pt.PT_ERR_CAPACITY and "max_hits" in str(ei.value)
        bad = ev.layer.copy()
        bad[5] = 10
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_load_hits(ev.x, ev.y, ev.z, bad)
        assert ei.value.status == pt.PT_ERR_INVALID
        d = [torch.from_numpy(v).cuda() for v in (ev.x, ev.y, ev.z, bad)]
        ctx.pt_load_hits(*d)
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_build_doublets()
        assert ei.value.status == pt.PT_ERR_INVALID
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_load_batch([0, 5, 3], ev.x, ev.y, ev.z, ev.layer)
        assert ei.value.status in (pt.PT_ERR_INVALID, pt.PT_ERR_CAPACITY)
    # link and ntuplet capacities: the overflow is reported, never truncated silently
    ev2 = sim.generate(sim.PU50, 2052)
    for field, stage in (("max_links", "pt_connect_cells"), ("max_ntuplets", "pt_find_ntuplets")):
        cap2 = dict(PU_CAP, **{field: 50})
        with pt.Context(cuts=cuts, capacity=cap2) as c2:
            c2.pt_load_hits(ev2.x, ev2.y, ev2.z, ev2.layer)
            with pytest.raises(pt.PtError) as ei:
                c2.pt_build_doublets()
                c2.pt_connect_cells()
                c2.pt_find_ntuplets()
                c2.pt_fit_tracks()
            assert ei.value.status == pt.PT_ERR_CAPACITY and field in str(ei.value)
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        # the context stays usable after errors
        small = sim.generate(sim.SINGLE_MUON_LIKE, 1001)
        hits, nh, tr, off = ctx.pt_reconstruct_batch([0, small.n_hits], small.x, small.y,
                                                     small.z, small.layer)
        ref = oracle.reconstruct(small.x, small.y, small.z, small.layer, cuts)
        assert np.array_equal(hits, oracle.survivors_hits(ref))


def test_bench_configuration_sampled(cuts):
    """The benchmark's launch configuration (64 PU200 events per batch, its capacity
    and binning): three events checked bit-exactly against the oracle, all events
    checked for canonical order, uniqueness and allowed layer chains."""
    import bench
    events = bench.make_events(bench.BATCH, seed0=bench.SEED0)
    off, x, y, z, layer = sim.concat(events)
    with pt.Context(cuts=cuts, capacity=bench.capacity()) as ctx:
        hits, nh, tracks, evoff = ctx.pt_reconstruct_batch(off, x, y, z, layer)
        hits, nh, tracks, evoff = (np.copy(v) for v in (hits, nh, tracks, evoff))
    from sim import truth
    allowed = set(truth.LAYER_PAIRS)
    for e, ev in enumerate(events):
        h = hits[evoff[e]:evoff[e + 1]]
        keys = [tuple(r) for r in h.tolist()]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
        for r, n in zip(h, nh[evoff[e]:evoff[e + 1]]):
            lay = ev.layer[r[:n]].tolist()
            assert all((u, v) in allowed for u, v in zip(lay[:-1], lay[1:]))
    for e in (0, len(events) // 2, len(events) - 1):
        ev = events[e]
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        sl = slice(evoff[e], evoff[e + 1])
        assert_ntuplets_equal(hits[sl], oracle.survivors_hits(ref), ref)
        assert_fits_close(tracks[sl], ref["fit"])


class _Hits:
    """Bare hit arrays in the Event layout that sim.concat reads."""

    def __init__(self, x, y, z, layer):
        self.x, self.y, self.z = (np.asarray(v, np.float32) for v in (x, y, z))
        self.layer = np.asarray(layer, np.uint8)
        self.n_hits = self.x.size


def _fan_event(sizes, seed=0):
    """Middle hits on layer 1, each crossed by n x n nearly collinear radial lines: n hits
    on layer 0 and n on layer 2 whose r-z slopes differ by 1e-4, so every (inner, outer)
    pair through the middle hit passes C1-C3 and the middle hit carries n*n links."""
    rng = np.random.default_rng(seed)
    x, y, z, lay = [], [], [], []
    for k, n in enumerate(sizes):
        phi = 0.4 + 0.9 * k
        z1 = -10.0 + 7.0 * k
        t0 = rng.uniform(-1, 1)
        pts = [(6.8, z1, 1)]
        for i in range(n):
            t = t0 + 1e-4 * i
            pts.append((2.9, z1 - t * (6.8 - 2.9), 0))
            pts.append((10.9, z1 + t * (10.9 - 6.8), 2))
        for r, zz, L in pts:
            x.append(r * np.cos(phi))
            y.append(r * np.sin(phi))
            z.append(zz)
            lay.append(L)
    return _Hits(x, y, z, lay)


def test_dense_middle_hits_many_links(cuts):
    """Middle hits with 64 (the in-kernel collection), 81 and 144 links: the second search
    pass, the per-source sort of a hit's links and the temporary copy it uses."""
    ev = _fan_event([8, 9, 12, 3])
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    h1 = ref["cell_outer"][ref["link_a"]]
    assert sorted(np.bincount(h1)[np.bincount(h1) > 0].tolist()) == [9, 64, 81, 144]
    with pt.Context(cuts=cuts, capacity=SMALL_CAP) as ctx:
        out = run_stages(ctx, [ev, sim.generate(sim.SINGLE_MUON_LIKE, 1100)])
        check_event(out, 0, ev, ref)
        n_links = out["n_links"]
        # the same batch through the captured whole-chain graph
        hits, nh, tr, eoff = ctx.pt_reconstruct_batch(*sim.concat(
            [ev, sim.generate(sim.SINGLE_MUON_LIKE, 1100)]))
    assert n_links == ref["link_a"].size + out["links"][0][out["links"][4] == 1].size
    assert_ntuplets_equal(hits[eoff[0]:eoff[1]], oracle.survivors_hits(ref), ref)


def test_poisson_batch_sampled(cuts):
    """The batch workload (64 events, pileup ~ Poisson(140) clipped to [20, 250], seeds
    5000+i) through the whole-chain graph at the benchmark's capacity: four events of
    different sizes (the smallest, the largest and two others) bit-exact against the
    oracle, every event in canonical order with allowed layer chains."""
    import bench
    pus = sim.batch_pileups(bench.CONFIG4_SEED0, bench.BATCH)
    events = [sim.pileup_event(bench.CONFIG4_SEED0 + i, int(p)) for i, p in enumerate(pus)]
    off, x, y, z, layer = sim.concat(events)
    with pt.Context(cuts=cuts, capacity=bench.capacity(bench.BATCH, 2048)) as ctx:
        dev = [torch.from_numpy(a).cuda() for a in (x, y, z, layer)]
        ctx.pt_enqueue_batch(off, *dev)
        hits, nh, evoff = (np.copy(v) for v in ctx.pt_get_ntuplets())
        tracks = ctx.pt_get_tracks()
    from sim import truth
    allowed = set(truth.LAYER_PAIRS)
    for e, ev in enumerate(events):
        h = hits[evoff[e]:evoff[e + 1]]
        keys = [tuple(r) for r in h.tolist()]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
        for r, n in zip(h, nh[evoff[e]:evoff[e + 1]]):
            lay = ev.layer[r[:n]].tolist()
            assert all((u, v) in allowed for u, v in zip(lay[:-1], lay[1:]))
    sizes = np.array([ev.n_hits for ev in events])
    for e in sorted({int(sizes.argmin()), int(sizes.argmax()), 7, 40}):
        ev = events[e]
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        sl = slice(evoff[e], evoff[e + 1])
        assert_ntuplets_equal(hits[sl], oracle.survivors_hits(ref), ref)
        assert_fits_close(tracks[sl], ref["fit"])


def _edge_event(rng, n_lines, cuts):
    """Tracks whose r-z lines start at z0 = +-z0max or have |slope| = cotmax, each nudged
    by a few float32 ulp either way, through the barrel layers and the disks (hits only
    where a line meets a layer inside its extent), on circles through the beam line with
    0.15 to 0.8 of the largest curvature (so the fitted charge is defined): the cells sit
    on the D2 and D3 edges, and with a few tracks per event most layers' r-z extents are
    a point or a thin box, the cases where the search windows' r-z reachability test has
    the least room."""
    z0max, cot = float(cuts["z0max"]), float(cuts["cotmax"])
    x, y, z, lay = [], [], [], []
    for _ in range(n_lines):
        phi = rng.uniform(-np.pi, np.pi)
        kap = rng.choice([-1.0, 1.0]) * rng.uniform(0.15, 0.8) * float(cuts["kmax"])
        turn = lambda r: phi + np.arcsin(0.5 * kap * r)  # noqa: E731
        if rng.random() < 0.5:
            z0 = rng.choice([-1.0, 1.0]) * z0max * (1 + rng.choice([-3, -1, 0, 1, 3]) * 6e-8)
            s = rng.uniform(-2.0, 2.0)
        else:
            z0 = rng.uniform(-z0max, z0max)
            s = rng.choice([-1.0, 1.0]) * cot * (1 + rng.choice([-3, -1, 0, 1, 3]) * 6e-8)
        for L, rl in enumerate(sim.events.BARREL_R):
            zz = z0 + s * rl
            if abs(zz) < sim.events.BARREL_ZMAX:
                x.append(rl * np.cos(turn(rl))), y.append(rl * np.sin(turn(rl)))
                z.append(zz), lay.append(L)
        for j, zd in enumerate(sim.events.DISK_Z):
            for side, base in ((1.0, 4), (-1.0, 7)):
                if s * side <= 0:
                    continue
                r = (side * zd - z0) / s
                if sim.events.DISK_RMIN <= r <= sim.events.DISK_RMAX:
                    x.append(r * np.cos(turn(r))), y.append(r * np.sin(turn(r)))
                    z.append(side * zd), lay.append(base + j)
    return _Hits(x, y, z, lay)


def test_cut_edge_lines_and_point_layers_match_oracle(small_ctx, cuts):
    rng = np.random.default_rng(606)
    events = [_edge_event(rng, n, cuts) for n in (1, 2, 3, 5, 8, 13, 40, 120)]
    out = run_stages(small_ctx, events)
    n_cells = 0
    for e, ev in enumerate(events):
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        n_cells += ref["cell_inner"].size
        check_event(out, e, ev, ref, edge_cases=True)
    assert n_cells > 100


def test_stage_ntuplets_follow_the_link_stage_form(cuts):
    """The stage-path ntuplet search follows the links as the last link stage left them:
    a gate switched on after a plain link stage does not change the plain result, and
    one switched off after a gated link stage does not change the gated result."""
    ev = sim.generate(sim.PU50, 2030, n_particles=600)
    batch = sim.concat([ev])
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    with pt.Context(cuts=cuts, capacity=PU_CAP) as ctx:
        ctx.pt_load_batch(*batch)
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_set_gate(*pt.default_gate())
        ctx.pt_find_ntuplets()
        plain = ctx.pt_get_ntuplets()[0]
        gated_graph = ctx.pt_reconstruct_batch(*batch)[0]
        ctx.pt_load_batch(*batch)
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_set_gate(None, 0.0)
        ctx.pt_find_ntuplets()
        gated_stage = ctx.pt_get_ntuplets()[0]
    assert_ntuplets_equal(plain, oracle.survivors_hits(ref), ref)
    assert np.array_equal(gated_stage, gated_graph)
    assert not np.array_equal(gated_graph, plain)
