"""Skip-layer (gap) doublets on the GPU: the chain over the extended layer-pair table
(the 13 chain pairs plus the 10 two-step pairs) against the oracle's orc_reconstruct_pairs
on events whose sensors miss 10 % of the crossings, element by element (cells, links with
their float32 quality, ntuplet candidates, cleaned ntuplets, fits); the default table
restored afterwards gives the default chain again; invalid tables are refused."""

import dataclasses

import numpy as np
import pytest

import oracle
import sim
from parity import assert_fits_close, assert_ntuplets_equal, cell_set, oracle_link_triples

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402
from test_gpu_parity import run_stages  # noqa: E402

FULL = oracle.DEFAULT_PAIRS + oracle.gap_pairs()
CAP = pt.default_capacity(max_events=2, hits_per_event=32768, cells_per_event=1 << 21,
                          links_per_event=1 << 18, ntuplets_per_event=1 << 17, phi_bins=1024)


def _check(out, e, ref):
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
    assert got_c == exp_c and int(m.sum()) == ref["nt_n"].size
    nth, ntn, evoff = out["nt"]
    sl = slice(evoff[e], evoff[e + 1])
    assert_ntuplets_equal(nth[sl], oracle.survivors_hits(ref), ref)
    assert_fits_close(out["tracks"][sl], ref["fit"])


def test_gap_pairs_match_oracle(cuts_low_pt):
    cfg = dataclasses.replace(sim.PU50, hit_eff=0.9)
    events = [sim.generate(cfg, 2400 + i) for i in range(2)]
    with pt.Context(cuts=cuts_low_pt, capacity=CAP) as ctx:
        ctx.pt_set_layer_pairs(FULL)
        out = run_stages(ctx, events)
        for e, ev in enumerate(events):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts_low_pt, pairs=FULL)
            _check(out, e, ref)
        # the whole-batch graph with the extended table
        hits, nh, tr, eoff = ctx.pt_reconstruct_batch(*sim.concat(events))
        for e, ev in enumerate(events):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts_low_pt, pairs=FULL)
            assert_ntuplets_equal(hits[eoff[e]:eoff[e + 1]], oracle.survivors_hits(ref), ref)
        # back to the default table
        ctx.pt_set_layer_pairs(None)
        out = run_stages(ctx, events)
        for e, ev in enumerate(events):
            _check(out, e, oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts_low_pt))


def test_gap_pairs_pu200(cuts):
    """A PU200 event (10 % of crossings lost) with the extended table: cleaned ntuplets
    bit-exact, and more of them than with the default table."""
    ev = sim.generate(dataclasses.replace(sim.PU200, hit_eff=0.9), 3150)
    cap = pt.default_capacity(max_events=1, hits_per_event=65536, cells_per_event=8 << 20,
                              links_per_event=1 << 20, ntuplets_per_event=1 << 19, phi_bins=2048)
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        ctx.pt_set_layer_pairs(FULL)
        hits, nh, tr, eoff = (np.copy(v) for v in ctx.pt_reconstruct_batch(
            [0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer))
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, pairs=FULL)
        assert_ntuplets_equal(hits, oracle.survivors_hits(ref), ref)
        assert_fits_close(tr, ref["fit"])
        ctx.pt_set_layer_pairs(None)
        h_def = ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)[0]
    assert hits.shape[0] > h_def.shape[0]


@pytest.mark.parametrize("bad", [[(0, 0)], [(0, 10)], [(-1, 2)], [(0, 1), (0, 1)],
                                 [(1, 0), (0, 1)], [(0, 1)] * 65,
                                 [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)],
                                 [(0, k) for k in range(1, 8)]])
def test_invalid_tables_are_refused(cuts, bad):
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_set_layer_pairs(bad)
        assert ei.value.status == pt.PT_ERR_INVALID
