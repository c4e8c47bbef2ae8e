"""Per-kernel tracing of the stage calls (pt_set_tracing / pt_get_trace): every kernel of
a stage run is reported once with a positive device time; the whole-batch graph is
never traced; results do not change with tracing on."""

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
STAGE_KERNELS = {"k_clear": 1, "k_bin_count": 1, "scan": 3, "k_bin_scatter": 1,
                 "k_doublets": 1, "k_connect": 1, "k_link_targets": 1, "k_find_ntuplets": 1,
                 "k_bucket_count": 1, "k_bucket_scatter": 1, "k_bucket_sort": 1,
                 "k_dedup_min": 1, "k_dedup_alive": 1, "k_dedup_triplets": 1, "k_compact": 1,
                 "k_event_offsets": 1, "k_fit": 1}


def _stages(ctx, ev):
    ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
    ctx.pt_build_doublets()
    ctx.pt_connect_cells()
    ctx.pt_find_ntuplets()
    ctx.pt_fit_tracks()
    return ctx.pt_get_ntuplets()


def test_trace_of_one_stage_run(cuts):
    ev = sim.generate(sim.PU50, 2300)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        with pytest.raises(pt.PtError) as ei:
            ctx.pt_get_trace()
        assert ei.value.status == pt.PT_ERR_INVALID
        ref = _stages(ctx, ev)
        ctx.pt_set_tracing(True)
        got = _stages(ctx, ev)
        tr = ctx.pt_get_trace()
        assert tr.pop("k_export_ntuplets")[1] >= 1  # the getter's export kernel
        assert {k: n for k, (_, n) in tr.items()} == STAGE_KERNELS
        assert all(ms > 0 for ms, _ in tr.values())
        assert ctx.pt_get_trace() == {}           # totals are cleared by a read
        ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
        assert ctx.pt_get_trace() == {}           # the graph is never traced
        ctx.pt_set_tracing(False)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
