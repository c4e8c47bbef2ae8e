"""Small single-threaded driver of the chain for kernel profilers (ncu).

Runs the stage path (load, doublets, links, ntuplets, fit, and optionally the
broken-line refit, vertices and raw data -> hits) on a batch of synthetic PU200 events
a few times, on one stream, with no autotuning, no worker threads and nothing else on
the GPU, and prints the per-kernel times of the last repetition.  A kernel's n-th
launch is its (n-1)-th repetition.

  python -m paper_2501_05520_gb300.profile_chain --events 8 --reps 3 [--gated]
         [--fishbone] [--overlap 0.2] [--extra] [--phi-bins 2048] [--blocks-per-sm 8]
         [--search-blocks-per-sm 8]
"""

from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed0", type=int, default=3000)
    ap.add_argument("--gated", action="store_true")
    ap.add_argument("--fishbone", action="store_true")
    ap.add_argument("--overlap", type=float, default=0.0,
                    help="fraction of crossings that also cross an overlapping sensor")
    ap.add_argument("--extra", action="store_true",
                    help="also run the refit, the vertices and raw data -> hits")
    ap.add_argument("--phi-bins", type=int, default=2048)
    ap.add_argument("--blocks-per-sm", type=int, default=8)
    ap.add_argument("--search-blocks-per-sm", type=int, default=8)
    a = ap.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2501_05520_gb300 as pt
    import sim

    import dataclasses
    cfg = dataclasses.replace(sim.PU200, overlap=a.overlap)
    events = [sim.generate(cfg, a.seed0 + i) for i in range(a.events)]
    off, x, y, z, layer = sim.concat(events)
    dev = torch.device("cuda", 0)
    d = [torch.from_numpy(v).to(dev) for v in (x, y, z, layer)]
    cap = pt.default_capacity(max_events=a.events, hits_per_event=65536,
                              cells_per_event=6_000_000 if a.overlap > 0 else 3_500_000, links_per_event=262_144,
                              ntuplets_per_event=196_608, phi_bins=a.phi_bins)
    with pt.Context(capacity=cap, device=0) as ctx:
        ctx.pt_set_launch(a.blocks_per_sm, a.search_blocks_per_sm)
        if a.gated:
            ctx.pt_set_gate(*pt.default_gate())
        if a.fishbone:
            ctx.pt_set_fishbone(True)
        raw = None
        if a.extra:
            from sim import pixels
            words = pixels.digitize(events[0])[0]
            roff, allw = pixels.concat_raw([words] * a.events)
            raw = (roff, torch.from_numpy(allw.view("int64")).to(dev))
            ctx.pt_set_modules()
        for r in range(a.reps):
            if r == a.reps - 1:
                ctx.pt_set_tracing(True)
            ctx.pt_load_batch(off, *d)
            counts = dict(cells=ctx.pt_build_doublets(), links=ctx.pt_connect_cells(),
                          ntuplets=ctx.pt_find_ntuplets(), tracks=ctx.pt_fit_tracks())
            if a.extra:
                ctx.pt_refit_broken_line(0.02, 0.02)
                ctx.pt_find_vertices()
                ctx.pt_load_raw(*raw)
        tr = ctx.pt_get_trace()
    torch.cuda.synchronize()
    print(counts)
    for k, (ms, n) in tr.items():
        print(f"{k:24s} {ms / n:8.4f} ms x {n}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
