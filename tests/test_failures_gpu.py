"""Failure detection in the forms that fault, trap or hang no GPU: a bounded device-side
wait made to run out (the gate's tensor-core waits with a limit of one cycle) comes
back as PT_ERR_TIMEOUT and leaves the context usable; a workspace larger than the
device is refused with PT_ERR_NOMEM and leaves the device usable; clients that abandon
their tickets leave the server's other results and its shutdown intact."""

import ctypes

import numpy as np
import pytest

import sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

CAP = pt.default_capacity(max_events=2, hits_per_event=16384, cells_per_event=1 << 20,
                          links_per_event=1 << 17, ntuplets_per_event=1 << 16)


def _gated_run(ctx, ev):
    ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
    ctx.pt_build_doublets()
    n = ctx.pt_connect_cells()
    ctx.pt_find_ntuplets()
    return n, ctx.pt_get_ntuplets()[0].copy()


def test_gate_wait_runs_out(cuts):
    ev = sim.generate(sim.PU50, 2500)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_gate(*pt.default_gate())
        n_ref, h_ref = _gated_run(ctx, ev)
        ctx.pt_set_wait_limit(1)
        ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
        ctx.pt_build_doublets()
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_connect_cells()
        assert ei.value.status == pt.PT_ERR_TIMEOUT
        assert "gate" in pt.lib().pt_last_error().decode()
        # the whole-batch graph reports it too
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
        assert ei.value.status == pt.PT_ERR_TIMEOUT
        # the default limit again: the same links and ntuplets as before
        ctx.pt_set_wait_limit(1 << 31)
        n, h = _gated_run(ctx, ev)
        assert n == n_ref and np.array_equal(h, h_ref)


def test_gate_score_wait_runs_out(cuts):
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_gate(*pt.default_gate())
        feat = torch.rand((1000, 12), device="cuda")
        out = torch.empty(1000, device="cuda")
        ctx.pt_gate_score(feat, out)
        ref = out.clone()
        ctx.pt_set_wait_limit(1)
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_gate_score(feat, out)
        assert ei.value.status == pt.PT_ERR_TIMEOUT
        ctx.pt_set_wait_limit(1 << 31)
        ctx.pt_gate_score(feat, out)
        assert torch.equal(out, ref)


def test_workspace_larger_than_the_device(cuts):
    free, total = torch.cuda.mem_get_info()
    cap = dict(pt.default_capacity(max_events=1, hits_per_event=1 << 20,
                                   cells_per_event=(1 << 32) - 2,
                                   links_per_event=(1 << 32) - 2, ntuplets_per_event=1 << 20))
    need = pt.pt_workspace_size(cap)
    assert need > total
    h = ctypes.c_void_p(None)
    st = pt.lib().pt_create(ctypes.byref(pt.PtGeometry(3.8)),
                            ctypes.byref(pt.PtCuts(*(float(cuts[k]) for k, _ in pt.PtCuts._fields_))),
                            ctypes.byref(pt._cap(cap)), 0, None, 0, None, ctypes.byref(h))
    assert st == pt.PT_ERR_NOMEM and not h.value
    assert "workspace" in pt.lib().pt_last_error().decode()
    # the device is still usable
    ev = sim.generate(sim.SINGLE_MUON_LIKE, 1000)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        hits, _, _, _ = ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
    assert hits.shape[0] > 0


def test_abandoned_tickets(cuts):
    """Half of the clients submit and never poll: the other half get the results their
    events give alone, statistics count every completed request, and the server shuts
    down with the abandoned results still held."""
    events = [sim.pileup_event(6500 + i, pu) for i, pu in enumerate((60, 120, 40, 150, 80, 30))]
    with pt.Context(cuts=cuts, capacity=pt.default_capacity(
            max_events=1, hits_per_event=65536, cells_per_event=4 << 20,
            links_per_event=1 << 20, ntuplets_per_event=1 << 19)) as ctx:
        alone = [ctx.pt_reconstruct_batch([0, e.n_hits], e.x, e.y, e.z, e.layer)[0].copy()
                 for e in events]
    srv = pt.Server(cuts=cuts, budget_bytes=2 << 30, slots=2)
    tickets = [srv.pt_submit(e.x, e.y, e.z, e.layer) for e in events]
    for i in (1, 3, 5):  # clients 0, 2, 4 walk away
        h, _, _ = srv.pt_poll(tickets[i], -1)
        assert np.array_equal(h, alone[i])
    # the abandoned requests complete on the device all the same
    for _ in range(200):
        if srv.pt_server_stats()["n_done"] == len(events):
            break
        import time
        time.sleep(0.01)
    assert srv.pt_server_stats()["n_done"] == len(events)
    srv.close()  # returns with three results never collected
    with pt.Server(cuts=cuts, budget_bytes=2 << 30, slots=2) as srv2:
        t = srv2.pt_submit(events[0].x, events[0].y, events[0].z, events[0].layer)
        assert np.array_equal(srv2.pt_poll(t, -1)[0], alone[0])
