"""Autotuner: the azimuthal bin count and the launch sizes change the speed only, never
the results; pt_autotune picks the fastest measured candidate; the JSON cache."""

import numpy as np
import pytest

import sim

torch = pytest.importorskip("torch")

import paper_2501_05520_gb300 as pt  # noqa: E402
from paper_2501_05520_gb300 import autotune  # noqa: E402

gpu = pytest.mark.gpu
needs_cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def test_cache_store_and_load(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert autotune._load(p) == {}
    autotune._store(p, "a", dict(phi_bins=512))
    autotune._store(p, "b", dict(phi_bins=1024))
    assert autotune._load(p) == {"a": {"phi_bins": 512}, "b": {"phi_bins": 1024}}
    (tmp_path / "bad.json").write_text("{not json")
    assert autotune._load(str(tmp_path / "bad.json")) == {}


def _batch():
    evs = [sim.generate(sim.PU200, 5100), sim.generate(sim.PU50, 5101),
           sim.generate(sim.SINGLE_MUON_LIKE, 5102)]
    return evs, sim.concat(evs)


def _cap(phi_bins):
    return pt.default_capacity(max_events=3, hits_per_event=65536, cells_per_event=4 << 20,
                               links_per_event=1 << 20, ntuplets_per_event=1 << 19,
                               phi_bins=phi_bins)


@gpu
@needs_cuda
def test_results_independent_of_bins_and_launch(cuts):
    _, (off, x, y, z, layer) = _batch()
    ref = None
    for phi_bins, bps, sbps in ((16, 1, 1), (256, 4, 5), (1024, 2, 8), (4096, 32, 32)):
        with pt.Context(cuts=cuts, capacity=_cap(phi_bins)) as ctx:
            ctx.pt_set_launch(bps, sbps)
            h, n, t, eo = ctx.pt_reconstruct_batch(off, x, y, z, layer)
            got = (h.tobytes(), n.tobytes(), t.tobytes(), eo.tobytes())
        assert h.shape[0] > 1000
        if ref is None:
            ref = got
        assert got == ref, (phi_bins, bps, sbps)


@gpu
@needs_cuda
def test_set_launch_rejects_bad_sizes(cuts):
    with pt.Context(cuts=cuts, capacity=_cap(256)) as ctx:
        for a, b in ((0, 5), (4, 0), (33, 5)):
            with pytest.raises(pt.PtError) as ei:
                ctx.pt_set_launch(a, b)
            assert ei.value.status == pt.PT_ERR_INVALID


@gpu
@needs_cuda
def test_autotune_picks_fastest_and_caches(cuts, tmp_path):
    _, (off, x, y, z, layer) = _batch()
    cand = dict(phi_bins=(64, 512), blocks_per_sm=(2, 4), search_blocks_per_sm=(5,))
    path = str(tmp_path / "tune.json")
    r = autotune.tuned(off, x, y, z, layer, _cap(256), cuts=cuts, path=path, reps=3, **cand)
    assert r["source"] == "measured"
    assert len(r["table"]) == 4 and all(v > 0 for v in r["table"].values())
    best = f"{r['phi_bins']}x{r['blocks_per_sm']}x{r['search_blocks_per_sm']}"
    assert r["table"][best] == min(r["table"].values())
    again = autotune.tuned(off, x, y, z, layer, _cap(256), cuts=cuts, path=path, **cand)
    assert again["source"] == "cache"
    assert {k: again[k] for k in ("phi_bins", "blocks_per_sm", "search_blocks_per_sm")} == \
        {k: r[k] for k in ("phi_bins", "blocks_per_sm", "search_blocks_per_sm")}
    with pytest.raises(pt.PtError):
        pt.pt_autotune(off, x, y, z, layer, _cap(256), phi_bins=(), cuts=cuts)
