"""Fishbone step on the GPU against the oracle's fishbone step, on events whose
sensors overlap (a second hit on the same layer for 20 % of the crossings): cells, the
links that remain (with their float32 quality), ntuplet candidates, cleaned ntuplets and
fits bit-exact (fits within the parity tolerance); the same with the skip-layer pairs,
through the whole-batch graph, with the learned gate, and switched off again."""

import dataclasses

import numpy as np
import pytest

import oracle
import sim
from oracle import gate as ogate
from parity import assert_ntuplets_equal, drop_near, near_hits

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402
from test_gap_gpu import _check  # noqa: E402
from test_gate_gpu import OUT_SCALE, TAU_BAND, _weights  # noqa: E402
from test_gpu_parity import run_stages  # noqa: E402

OVERLAP = dataclasses.replace(sim.PU50, overlap=0.2)
FULL = oracle.DEFAULT_PAIRS + oracle.gap_pairs()
CAP = pt.default_capacity(max_events=2, hits_per_event=32768, cells_per_event=1 << 21,
                          links_per_event=1 << 18, ntuplets_per_event=1 << 17, phi_bins=1024)


def test_fishbone_matches_oracle(cuts):
    events = [sim.generate(OVERLAP, 4200 + i) for i in range(2)]
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_fishbone(True)
        out = run_stages(ctx, events)
        n_ref = 0
        for e, ev in enumerate(events):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, fishbone=True)
            off = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
            assert ref["link_a"].size < off["link_a"].size  # the step removes links here
            _check(out, e, ref)
            n_ref += ref["link_a"].size
        assert out["n_links"] == n_ref
        # the whole-batch graph runs the step too
        hits, nh, tr, eoff = ctx.pt_reconstruct_batch(*sim.concat(events))
        for e, ev in enumerate(events):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, fishbone=True)
            assert_ntuplets_equal(hits[eoff[e]:eoff[e + 1]], oracle.survivors_hits(ref), ref)
        # switched off: the default chain again
        ctx.pt_set_fishbone(False)
        out = run_stages(ctx, events)
        for e, ev in enumerate(events):
            _check(out, e, oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts))


def test_fishbone_with_skip_layer_pairs(cuts_low_pt):
    cfg = dataclasses.replace(OVERLAP, hit_eff=0.9)
    events = [sim.generate(cfg, 4210 + i) for i in range(2)]
    with pt.Context(cuts=cuts_low_pt, capacity=CAP) as ctx:
        ctx.pt_set_layer_pairs(FULL)
        ctx.pt_set_fishbone(True)
        out = run_stages(ctx, events)
        for e, ev in enumerate(events):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts_low_pt, pairs=FULL,
                                     fishbone=True)
            _check(out, e, ref)


def test_fishbone_after_the_gate(cuts):
    """Gate and fishbone: the step reads the links the gate keeps.  Ntuplets sharing a
    hit with a link in the gate's threshold band (or a near-threshold cut decision) are
    excluded on both sides, as in the gated parity test."""
    ev = sim.generate(OVERLAP, 4220)
    w = _weights(4, OUT_SCALE)
    ref0 = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    ci, co = ref0["cell_inner"], ref0["cell_outer"]
    h0, h1, h2 = ci[ref0["link_a"]], co[ref0["link_a"]], co[ref0["link_b"]]
    F = ogate.features(ev.x, ev.y, ev.z, ev.layer, h0, h1, h2, cuts)
    s = ogate.forward(w, F.astype(np.float32), bf16=True)
    tau = float(np.quantile(s, 0.4))
    keep = s >= tau
    near = np.abs(s - tau) <= TAU_BAND
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_gate(w, tau)
        ctx.pt_set_fishbone(True)
        hits, nh, tr, eoff = (np.copy(v) for v in ctx.pt_reconstruct_batch(
            [0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer))
    ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, link_keep=keep, fishbone=True)
    band = set(h0[near].tolist()) | set(h1[near].tolist()) | set(h2[near].tolist())
    band |= near_hits(ref)
    exp_nt = drop_near(oracle.survivors_hits(ref), band)
    got_nt = drop_near(hits, band)
    assert exp_nt.shape[0] > 0.8 * oracle.survivors_hits(ref).shape[0]
    assert np.array_equal(got_nt, exp_nt)


def test_set_fishbone_refuses_other_values(cuts):
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        with pytest.raises(pt.PtError) as ei:
            pt._check(pt.lib().pt_set_fishbone(ctx.handle, 2))
        assert ei.value.status == pt.PT_ERR_INVALID
