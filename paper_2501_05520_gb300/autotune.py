"""Measured choice of the azimuthal bin count and the launch sizes, with a JSON cache.

The chain's results do not depend on these three numbers (the binning only narrows the
candidate search, the persistent kernels are grid-stride loops), but its speed does, and
the best values move with the event size, the batch size and the GPU.  `tuned()` times
every candidate combination on a sample batch through pt_autotune (CUDA events around
the whole-chain graph, median of `reps` launches) and remembers the winner per
(GPU, sample shape, capacity, candidate lists) in a JSON file:

  $PTCA_TUNE_CACHE, else ~/.cache/paper_2501_05520_gb300/tune.json

  python -m paper_2501_05520_gb300.autotune --events 64   # PU200 sample, seeds 3000+
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

PHI_BINS = (64, 128, 256, 512, 1024, 2048)
BLOCKS_PER_SM = (2, 4, 8)
SEARCH_BLOCKS_PER_SM = (3, 5, 8)


def cache_path() -> str:
    p = os.environ.get("PTCA_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2501_05520_gb300", "tune.json")


def _gpu_id(device: int) -> str:
    import torch
    prop = torch.cuda.get_device_properties(device)
    return f"{prop.name}|sm{prop.major}{prop.minor}|{prop.multi_processor_count}"


def cache_key(device: int, offsets, capacity: dict, cuts: dict, candidates: tuple) -> str:
    """GPU, library build, sample shape (events, hits), capacity without phi_bins, cuts and
    candidate lists: a rebuilt library or another workload is measured afresh."""
    import paper_2501_05520_gb300 as pt
    off = np.asarray(offsets, np.int64)
    st = os.stat(pt.LIB_PATH)
    cap = {k: int(v) for k, v in sorted(capacity.items()) if k != "phi_bins"}
    desc = json.dumps(dict(gpu=_gpu_id(device), lib=[st.st_size, st.st_mtime_ns],
                           events=int(off.size - 1), hits=int(off[-1]),
                           cap=cap, cuts={k: float(v) for k, v in sorted(cuts.items())},
                           cand=[list(c) for c in candidates]), sort_keys=True)
    return hashlib.sha1(desc.encode()).hexdigest()[:16]


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, entry: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    data = _load(path)
    data[key] = entry
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(offsets, x, y, z, layer, capacity: dict, cuts: dict | None = None, device: int = 0,
          phi_bins=PHI_BINS, blocks_per_sm=BLOCKS_PER_SM,
          search_blocks_per_sm=SEARCH_BLOCKS_PER_SM, reps: int = 3, path: str | None = None,
          refresh: bool = False) -> dict:
    """Best {phi_bins, blocks_per_sm, search_blocks_per_sm} for this sample batch, from the
    cache or measured (then stored).  `source` says which; `table` holds every median."""
    import paper_2501_05520_gb300 as pt
    cuts = dict(cuts or pt.default_cuts())
    cand = (tuple(phi_bins), tuple(blocks_per_sm), tuple(search_blocks_per_sm))
    path = path or cache_path()
    key = cache_key(device, offsets, capacity, cuts, cand)
    if not refresh:
        hit = _load(path).get(key)
        if hit:
            return dict(hit, source="cache")
    t0 = time.perf_counter()
    res = pt.pt_autotune(offsets, x, y, z, layer, capacity, phi_bins=phi_bins,
                         blocks_per_sm=blocks_per_sm, search_blocks_per_sm=search_blocks_per_sm,
                         reps=reps, cuts=cuts, device=device)
    res["seconds"] = round(time.perf_counter() - t0, 2)
    res["gpu"] = _gpu_id(device)
    try:
        _store(path, key, res)
    except OSError:
        pass  # an unwritable cache only costs a re-measurement
    return dict(res, source="measured")


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import paper_2501_05520_gb300 as pt
    import sim
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--seed", type=int, default=3000)
    ap.add_argument("--refresh", action="store_true")
    a = ap.parse_args(argv)
    events = [sim.generate(sim.PU200, a.seed + i) for i in range(a.events)]
    off, x, y, z, layer = sim.concat(events)
    cap = pt.default_capacity(max_events=a.events, hits_per_event=49152,
                              cells_per_event=3_500_000, links_per_event=262_144,
                              ntuplets_per_event=196_608)
    print(json.dumps(tuned(off, x, y, z, layer, cap, refresh=a.refresh)))


if __name__ == "__main__":
    main()
