"""The debug build on the GPU: the whole chain (plain, gated, skip-layer pairs with the
fishbone step, the whole-batch graph) runs with every device-side bounds check in force
and none of them fires (a failing check turns the next synchronising call into
PT_ERR_INTERNAL), and the cleaned ntuplets equal the oracle's; a failure recorded by
pt_debug_inject is reported and cleared by the next load.  It runs in a child process,
which loads the debug library (PT_DEBUG=1)."""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import dataclasses, sys
    sys.path.insert(0, "tests")
    import numpy as np
    import oracle, sim
    import paper_2501_05520_gb300 as pt
    from parity import assert_ntuplets_equal
    assert pt.lib().pt_debug_build() == 1
    cuts = pt.default_cuts()
    cap = pt.default_capacity(max_events=4, hits_per_event=65536, cells_per_event=6 << 20,
                              links_per_event=1 << 20, ntuplets_per_event=1 << 19)
    full = pt.DEFAULT_PAIRS + pt.gap_pairs()
    pu200 = sim.generate(sim.PU200, 3300)
    pu50 = [sim.generate(dataclasses.replace(sim.PU50, overlap=0.2, hit_eff=0.9), 3310 + i)
            for i in range(3)]
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        # stage path, plain form
        ctx.pt_load_batch(*sim.concat([pu200]))
        ctx.pt_build_doublets(); ctx.pt_connect_cells(); ctx.pt_find_ntuplets()
        ctx.pt_fit_tracks()
        hits = ctx.pt_get_ntuplets()[0]
        ref = oracle.reconstruct(pu200.x, pu200.y, pu200.z, pu200.layer, cuts)
        assert_ntuplets_equal(hits, oracle.survivors_hits(ref), ref)
        # gated form through the graph
        ctx.pt_set_gate(*pt.default_gate())
        ctx.pt_reconstruct_batch(*sim.concat([pu200]))
        ctx.pt_set_gate(None, 0.0)
        # skip-layer pairs and the fishbone step through the graph
        ctx.pt_set_layer_pairs(full)
        ctx.pt_set_fishbone(True)
        hits, nh, tr, eoff = ctx.pt_reconstruct_batch(*sim.concat(pu50))
        for e, ev in enumerate(pu50):
            ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts, pairs=full, fishbone=True)
            assert_ntuplets_equal(hits[eoff[e]:eoff[e + 1]], oracle.survivors_hits(ref), ref)
        # the reporting path: a recorded failure comes back as PT_ERR_INTERNAL naming the
        # check, and the next load clears it
        ctx.pt_debug_inject(7)
        try:
            ctx.pt_get_ntuplets()
            raise AssertionError("no error reported")
        except pt.PtError as e:
            assert e.status == pt.PT_ERR_INTERNAL and "check 7" in str(e), e
        ctx.pt_reconstruct_batch(*sim.concat(pu50))
    print("debug chain ok")
""")


def test_debug_chain_checks_pass_and_matches_oracle():
    from paper_2501_05520_gb300 import build as pbuild
    pbuild.build(debug=True)
    env = dict(os.environ, PT_DEBUG="1")
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "debug chain ok" in res.stdout
