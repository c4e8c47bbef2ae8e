#!/usr/bin/env python3
"""Benchmark of the pixel-track CA chain on GB300: PU200 events/s.

One step = the whole chain (load + bin, doublets, links, ntuplets + cleaning, fit) over
one batch of BATCH synthetic PU200 events.  `value` is timed with CUDA events on the
library's stream with the inputs already in device memory; L2 is flushed (256 MB write)
before every step, outside the step's events.  `e2e` is the same metric through the
public C ABI call pt_reconstruct_batch with pinned host buffers (host->device copies and
the device->host read of the results inside the timed region), from two host threads
with a context each, so that one batch's copies overlap the other's kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica on its own GPU (events are independent,
no collective on the data path); rank 0 prints one JSON line.  `--impl reference`
times the CPU oracle on the host cores on the same workload.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sim  # noqa: E402

BATCH = 64
SEED0 = 3000
METRIC = "PU200 events/s on 1 GB300, plain CA vs MLP-gated (eff ≥ plain−0.5%); p99 ms"
WORKLOAD = ("PU200: 10k helices/event (1/pT~U[0.1,2] GeV^-1, |eta|<2.5, z0~N(0,5cm)), "
            "4 barrel layers + 2x3 disks, 2% noise, ~41k hits/event; plain CA")
FLUSH_BYTES = 256 << 20
TRACE_STEPS = 5      # extra stage-path steps with per-kernel CUDA events (after the timing)
E2E_THREADS = 3      # host threads of the end-to-end leg (3 measured fastest of 1..4)
CONFIG4_SEED0 = 5000  # batch workload: 64 events, pileup ~ Poisson(140) clipped to [20, 250]

# DRAM traffic per event of the main kernels from one ncu capture (8 PU200 events per
# launch, profiles/), valid only while the kernel's sources hash to the recorded value.
NCU_TRAFFIC = {
    "k_doublets": {"bytes_per_event": 24503712, "issue_active_pct": 58.4,
                   "warp_inst_per_event": 25200120, "sha": "2a8aa9a0d737"},
    "k_connect": {"bytes_per_event": 22363520, "issue_active_pct": 57.7,
                  "warp_inst_per_event": 45554002, "sha": "0d56a924773e"},
    "k_link_targets": {"bytes_per_event": 14528864, "issue_active_pct": 19.2,
                       "warp_inst_per_event": 840076, "sha": "0d56a924773e"},
    "k_find_ntuplets": {"bytes_per_event": 35716608, "issue_active_pct": 19.5,
                        "warp_inst_per_event": 2328577, "sha": "e73b2d03adb5"},
}
SMS, SCHEDULERS_PER_SM = 152, 4  # GB300: each scheduler issues one warp instruction a cycle


def make_events(n: int, seed0: int = SEED0):
    return [sim.generate(sim.PU200, seed0 + i) for i in range(n)]


def capacity(batch: int = BATCH, phi_bins: int = 1024) -> dict:
    import paper_2501_05520_gb300 as pt
    return pt.default_capacity(max_events=batch, hits_per_event=49152,
                               cells_per_event=3_500_000, links_per_event=262_144,
                               ntuplets_per_event=196_608, phi_bins=phi_bins)


# Algorithmic bytes of each step of the chain per batch (SURVEY-level accounting, the
# least each step must read or write whatever the layout): N hits, C cells, Lk links,
# T ntuplet candidates, I (cell, candidate) incidences, S cleaned ntuplets holding H hits.
#   A1 load + bin: 13 B/hit read (x, y, z, layer) + 20 B/hit written (x, y, z, r, index)
#   A2 doublets: 20 B/hit read (each hit staged once) + 10 B/cell written
#   A3 links: 8 B/cell read + 1 B/cell flag + 8 B/hit (per-hit lists) + 4 B/link written
#   A4 ntuplets: 4 B/link + 4 B/cell read + 29 B/candidate written
#   A5/A6 cleaning and order: 2 x 29 B/candidate + 4 B per incidence
#   A7 fit: 12 B per hit read + 36 B per track written
def stage_bytes(stage: str, c: dict) -> int:
    N, C, Lk, T = c["hits"], c["cells"], c["links"], c["candidates"]
    return {
        "A1": 13 * N + 20 * N,
        "A2": 20 * N + 10 * C,
        "A3": 9 * C + 8 * N + 4 * Lk,
        "A4": 4 * Lk + 4 * C + 29 * T,
        "A5A6": 58 * T + 4 * c["incidences"],
        "A7": 12 * c["survivor_hits"] + 36 * c["survivors"],
    }[stage]


# The step each traced kernel belongs to, and the steps each timed stage call covers.
KERNEL_STAGE = {"k_doublets": "A2", "k_connect": "A3", "k_link_targets": "A3",
                "k_find_ntuplets": "A4", "k_fit": "A7"}
CALL_STAGES = {"load": ("A1",), "doublets": ("A2",), "connect": ("A3",),
               "ntuplets": ("A4", "A5A6"), "fit": ("A7",)}


# Bytes of one launch of each main kernel in this library's own layout (every array the
# kernel touches, read or written once): reported beside the step accounting above.
def kernel_layout_bytes(kernel: str, c: dict) -> int | None:
    N, C, Lk, T = c["hits"], c["cells"], c["links"], c["candidates"]
    return {
        # hit (x,y,z,r) and bin 20 N; incoming segments 24 N; cells (inner, outer) 8 C and
        # their two link flags 2 C
        "k_doublets": 20 * N + 24 * N + 10 * C,
        # hit and bin 20 N, incoming segments 24 N; inner hit of each incoming cell 4 C;
        # links (source, target, quality, next) 16 Lk, list heads and out flags <= 5 Lk
        "k_connect": 44 * N + 4 * C + 21 * Lk,
        # link source and target 8 Lk (read), the source's outer hit and the target's
        # segment 12 Lk, target (write) and in flag 5 Lk
        "k_link_targets": 25 * Lk,
        # link sources (root search) 4 Lk, roots' flags and lists <= 10 Lk, link targets
        # and qualities 8 Lk; candidates (6 hits, 5 cells, n, q) 49 T
        "k_find_ntuplets": 22 * Lk + 49 * T,
    }.get(kernel)


def kernel_sources_sha(kernel: str) -> str:
    import hashlib
    src = {"k_doublets": "doublets.cu", "k_connect": "connect.cu", "k_link_targets": "connect.cu",
           "k_find_ntuplets": "ntuplets.cu"}[kernel]
    d = os.path.join(ROOT, "paper_2501_05520_gb300", "csrc")
    h = hashlib.sha1()
    for f in (src, "ptca_internal.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                p = [v.strip() for v in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _issue_roof(rec, events: int, launch_ms: float, clocks) -> dict | None:
    """The kernel against the instruction-issue roof: its warp instructions per launch
    (ncu count per event x events) over the launch time, against 152 SMs x 4 schedulers x
    one warp instruction per cycle at the SM clock seen during the timed steps (the
    largest, 2070 MHz, when none was sampled)."""
    if rec is None:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    inst = rec["warp_inst_per_event"] * events
    achieved = inst / (launch_ms / 1000.0) / 1e9
    peak = SMS * SCHEDULERS_PER_SM * mhz / 1000.0
    return {"warp_inst": inst, "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "Ginst/s", "frac": round(achieved / peak, 4), "sm_mhz": mhz}


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


def cpu_baseline(n_events: int | None = None, seed0: int = SEED0 + 500,
                 one_thread: bool = True) -> dict:
    """The oracle as it stands, one PU200 event per host thread (and, with one_thread,
    the first event alone on one thread before that)."""
    import oracle
    import paper_2501_05520_gb300 as pt
    cuts = pt.default_cuts()
    cores = os.cpu_count() or 1
    n = n_events or max(1, min(cores, 16))
    evs = make_events(n, seed0)
    oracle.build()
    dt1 = None
    if one_thread:
        t1 = time.perf_counter()
        oracle.reconstruct(evs[0].x, evs[0].y, evs[0].z, evs[0].layer, cuts)
        dt1 = time.perf_counter() - t1
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(cores, n)) as ex:
        list(ex.map(lambda e: oracle.reconstruct(e.x, e.y, e.z, e.layer, cuts), evs))
    dt = time.perf_counter() - t0
    out = {"value": n / dt, "unit": "events/s", "cores": min(cores, n), "kind": "oracle",
           "sample": f"{n} PU200 events (seeds {seed0}..{seed0 + n - 1}), one per thread, "
                     f"{platform.machine()} host, {dt:.1f} s", "host_cores": cores}
    if dt1 is not None:
        out["one_thread"] = {"value": 1.0 / dt1, "unit": "events/s",
                             "sample": f"event {seed0} alone, {dt1:.1f} s"}
    return out


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed0(rank: int) -> int:
    """First event seed of a rank: the replicas process disjoint synthetic event streams."""
    return SEED0 + rank * 100_000


def max_over_ranks(seconds: float, dist=None, device="cpu") -> float:
    """The job's time is its slowest rank's (no-op on one process)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, events_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank's events over the slowest rank's time."""
    return world * events_per_step * steps / seconds


def run_reference(args):
    rank, world, local = _dist_env()
    if rank != 0:
        return
    import paper_2501_05520_gb300 as pt  # noqa: F401  (cut constants only)
    cores = os.cpu_count() or 1
    per_step = max(1, min(cores, 16))
    for w in range(args.warmup):
        cpu_baseline(per_step, seed0=SEED0 + 700 + w * per_step, one_thread=False)
    vals = []
    t_all = 0.0
    for s in range(args.steps):
        r = cpu_baseline(per_step, seed0=SEED0 + s * per_step, one_thread=False)
        vals.append(r)
        t_all += per_step / r["value"]
    value = args.steps * per_step / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "events/s", "kind": "oracle",
                             "cores": vals[0]["cores"],
                             "sample": f"{per_step} PU200 events per step, one per thread"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(ctx, dbat, steps, flush, stream):
    """K steps of the stage path with CUDA events between the stages; L2 flushed
    before each step outside its events.  Returns per-step stage times (ms)."""
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)]
    for s_ in range(steps):
        flush.zero_()
        off, x, y, z, layer = dbat[s_ % 2]
        e = evs[s_]
        e[0].record(stream)
        ctx.pt_load_batch(off, x, y, z, layer)
        e[1].record(stream)
        ctx.pt_build_doublets(sync=False)
        e[2].record(stream)
        ctx.pt_connect_cells(sync=False)
        e[3].record(stream)
        ctx.pt_find_ntuplets(sync=False)
        e[4].record(stream)
        ctx.pt_fit_tracks(sync=False)
        e[5].record(stream)
    stream.synchronize()
    names = ["load", "doublets", "connect", "ntuplets", "fit"]
    stage = {n: [e[k].elapsed_time(e[k + 1]) for e in evs] for k, n in enumerate(names)}
    step = [e[0].elapsed_time(e[5]) for e in evs]
    return step, stage


def _e2e(pt, ctxs, host, B, steps, warmup):
    """`steps` batches through pt_reconstruct_batch from pinned host memory to host
    memory, split over one host thread per context; returns (wall seconds of the timed
    calls, ntuplets per batch)."""
    import threading
    import torch
    pin = [torch.from_numpy(a).pin_memory() for a in host[1:]]
    outs = []
    for c in ctxs:
        capn = int(c.capacity["max_ntuplets"])
        outs.append(dict(hits=torch.empty((capn, 6), dtype=torch.int32).pin_memory(),
                         nhits=torch.empty(capn, dtype=torch.uint8).pin_memory(),
                         tracks=torch.empty((capn, 36), dtype=torch.uint8).pin_memory(),
                         event_offsets=torch.empty(B + 1, dtype=torch.int64).pin_memory()))
    start = threading.Barrier(len(ctxs) + 1)
    done = threading.Barrier(len(ctxs) + 1)
    counts = [0] * len(ctxs)

    def worker(i):
        for _ in range(warmup):
            h, _, _, _ = ctxs[i].pt_reconstruct_batch(host[0], *pin, out=outs[i])
        counts[i] = int(h.shape[0]) if warmup else 0
        start.wait()
        for _ in range(steps // len(ctxs) + (1 if i < steps % len(ctxs) else 0)):
            ctxs[i].pt_reconstruct_batch(host[0], *pin, out=outs[i])
        done.wait()

    th = [threading.Thread(target=worker, args=(i,)) for i in range(len(ctxs))]
    for t in th:
        t.start()
    start.wait()
    t0 = time.perf_counter()
    done.wait()
    wall = time.perf_counter() - t0
    for t in th:
        t.join()
    return wall, max(counts)


def _config4(ctx, dev, flush, stream, steps, warmup, n_events):
    """The batch workload through the whole-chain CUDA graph (pt_enqueue_batch), inputs in
    device memory, L2 flushed before every step outside its events."""
    import torch
    pus = sim.batch_pileups(CONFIG4_SEED0, n_events)
    evs = [sim.pileup_event(CONFIG4_SEED0 + i, int(p)) for i, p in enumerate(pus)]
    off, *arrs = sim.concat(evs)
    d = [torch.from_numpy(a).to(dev) for a in arrs]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.pt_enqueue_batch(off, *d)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            ctx.pt_enqueue_batch(off, *d)
            e1.record(stream)
    stream.synchronize()
    ctx.pt_get_ntuplets()  # raises on any capacity or input error
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"value": n_events * steps / (sum(ms) / 1000.0), "unit": "events/s",
            "ms_per_step": statistics.mean(ms), "events_per_step": n_events,
            "hits_per_step": int(off[-1]),
            "workload": f"pileup ~ Poisson(140) in [20, 250], seeds {CONFIG4_SEED0}+i",
            "path": "whole-chain CUDA graph, device inputs"}


def _latency(pt, dev, n_timed: int = 40, warmup: int = 10) -> dict:
    """Per-event latency of single events through the public whole-chain call
    (pt_reconstruct_batch, host buffers in and out, one event per call): the
    50-particle barrel event, one PU50 event and one PU200 event; and PU50 events/s in
    batches of 64 through the captured graph with device inputs.  A single event's working
    set fits in L2, so these latencies are not HBM-bound."""
    import torch
    out = {}
    for name, cfg, seed0, hits in (("config1_barrel50", sim.SINGLE_MUON_LIKE, 1000, 4096),
                                   ("pu50_single", sim.PU50, 2000, 32768),
                                   ("pu200_single", sim.PU200, 3000, 65536)):
        evs = [sim.generate(cfg, seed0 + i) for i in range(warmup + n_timed)]
        cap = pt.default_capacity(max_events=1, hits_per_event=hits,
                                  cells_per_event=max(1 << 16, hits * 80),
                                  links_per_event=max(1 << 14, hits * 8),
                                  ntuplets_per_event=max(1 << 13, hits * 6), phi_bins=1024)
        with pt.Context(capacity=cap, device=dev.index or 0) as c:
            ms = []
            for i, e in enumerate(evs):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                c.pt_reconstruct_batch([0, e.n_hits], e.x, e.y, e.z, e.layer)
                t1 = time.perf_counter()
                if i >= warmup:
                    ms.append(1000.0 * (t1 - t0))
        out[name] = {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                     "mean_ms": float(np.mean(ms)), "events": len(ms),
                     "hits_per_event": float(np.mean([e.n_hits for e in evs])),
                     "path": "pt_reconstruct_batch, one event per call, host buffers"}
    # PU50 throughput in 64-event batches (graph, device inputs, L2 flushed per step)
    evs = [sim.generate(sim.PU50, 2000 + i) for i in range(64)]
    off, *arrs = sim.concat(evs)
    d = [torch.from_numpy(a).to(dev) for a in arrs]
    cap = pt.default_capacity(max_events=64, hits_per_event=16384, cells_per_event=400_000,
                              links_per_event=65536, ntuplets_per_event=65536, phi_bins=1024)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with pt.Context(capacity=cap, device=dev.index or 0) as c:
        s_ = c.stream
        with torch.cuda.stream(s_):
            for _ in range(3):
                c.pt_enqueue_batch(off, *d)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(20)]
            for e0, e1 in ev:
                flush.zero_()
                e0.record(s_)
                c.pt_enqueue_batch(off, *d)
                e1.record(s_)
        s_.synchronize()
        c.pt_get_ntuplets()
        ms = [a.elapsed_time(b) for a, b in ev]
    out["pu50_batch64"] = {"value": 64 * len(ms) / (sum(ms) / 1000.0), "unit": "events/s",
                           "ms_per_step": float(np.mean(ms)), "hits_per_step": int(off[-1]),
                           "path": "whole-chain CUDA graph, device inputs, L2 flushed per step"}
    return out


def _gap_form(pt, dev, flush, steps: int, n_events: int = 64) -> dict:
    """Skip-layer pairs: PU200 events whose sensors miss 10 % of the crossings (seeds
    3500+i), through the whole-chain graph with device inputs, with the default 13 pairs
    and with the 10 two-step pairs added; events/s and efficiency / fake rate against
    generator truth, a particle counting as reconstructable when it has a chain of >= 3
    hits on the extended table (the same denominator for both tables)."""
    import dataclasses
    import torch
    from sim import truth
    full = pt.DEFAULT_PAIRS + pt.gap_pairs()
    cfg = dataclasses.replace(sim.PU200, hit_eff=0.9)
    evs = [sim.generate(cfg, 3500 + i) for i in range(n_events)]
    off, *arrs = sim.concat(evs)
    d = [torch.from_numpy(a).to(dev) for a in arrs]
    cap = pt.default_capacity(max_events=n_events, hits_per_event=49152,
                              cells_per_event=8_500_000, links_per_event=524_288,
                              ntuplets_per_event=393_216, phi_bins=2048)
    out = {"workload": f"{n_events} PU200 events, 10 % of crossings lost, seeds 3500+i",
           "path": "whole-chain CUDA graph, device inputs, L2 flushed per step"}
    with pt.Context(capacity=cap, device=dev.index or 0) as c:
        c.pt_set_launch(8, 8)
        for name, pairs in (("default_pairs", None), ("gap_pairs", full)):
            c.pt_set_layer_pairs(pairs)
            s_ = c.stream
            with torch.cuda.stream(s_):
                for _ in range(2):
                    c.pt_enqueue_batch(off, *d)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                for e0, e1 in ev:
                    flush.zero_()
                    e0.record(s_)
                    c.pt_enqueue_batch(off, *d)
                    e1.record(s_)
            s_.synchronize()
            hits, nh, eoff = c.pt_get_ntuplets()
            ms = [a.elapsed_time(b) for a, b in ev]
            tot = dict(reco=0, matched=0.0, fake=0, nt=0)
            for e, evt in enumerate(evs):
                r = truth.rates_fast(hits[eoff[e]:eoff[e + 1]], evt.pid, evt.layer, pairs=full)
                tot["reco"] += r["n_reconstructable"]
                tot["matched"] += r["efficiency"] * r["n_reconstructable"]
                tot["fake"] += r["n_fake"]
                tot["nt"] += r["n_ntuplets"]
            out[name] = {"value": n_events * len(ms) / (sum(ms) / 1000.0), "unit": "events/s",
                         "ms_per_step": float(np.mean(ms)),
                         "efficiency": tot["matched"] / max(tot["reco"], 1),
                         "fake_rate": tot["fake"] / max(tot["nt"], 1), "n_ntuplets": tot["nt"]}
    return out


def _fishbone_form(pt, dev, flush, steps: int, n_events: int = 64) -> dict:
    """Fishbone step: PU200 events whose sensors overlap (a second hit on the same layer
    for 20 % of the crossings, seeds 3600+i), through the whole-chain graph with device
    inputs, with the step off and on; events/s, ntuplet candidates before cleaning, and
    efficiency / fake / duplicate rate against generator truth."""
    import dataclasses
    import torch
    from sim import truth
    cfg = dataclasses.replace(sim.PU200, overlap=0.2)
    evs = [sim.generate(cfg, 3600 + i) for i in range(n_events)]
    off, *arrs = sim.concat(evs)
    d = [torch.from_numpy(a).to(dev) for a in arrs]
    cap = pt.default_capacity(max_events=n_events, hits_per_event=65536,
                              cells_per_event=6_000_000, links_per_event=524_288,
                              ntuplets_per_event=393_216, phi_bins=2048)
    out = {"workload": f"{n_events} PU200 events, overlapping sensors on 20 % of the "
                       "crossings, seeds 3600+i",
           "path": "whole-chain CUDA graph, device inputs, L2 flushed per step"}
    with pt.Context(capacity=cap, device=dev.index or 0) as c:
        c.pt_set_launch(8, 8)
        for name, on in (("off", False), ("on", True)):
            c.pt_set_fishbone(on)
            s_ = c.stream
            with torch.cuda.stream(s_):
                for _ in range(2):
                    c.pt_enqueue_batch(off, *d)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                for e0, e1 in ev:
                    flush.zero_()
                    e0.record(s_)
                    c.pt_enqueue_batch(off, *d)
                    e1.record(s_)
            s_.synchronize()
            hits, nh, eoff = c.pt_get_ntuplets()
            n_cand = c.pt_get_candidates()[0].shape[0]
            ms = [a.elapsed_time(b) for a, b in ev]
            tot = dict(reco=0, matched=0.0, dup=0.0, fake=0, nt=0)
            for e, evt in enumerate(evs):
                r = truth.rates_fast(hits[eoff[e]:eoff[e + 1]], evt.pid, evt.layer)
                tot["reco"] += r["n_reconstructable"]
                tot["matched"] += r["efficiency"] * r["n_reconstructable"]
                tot["dup"] += r["duplicate_rate"] * r["n_reconstructable"]
                tot["fake"] += r["n_fake"]
                tot["nt"] += r["n_ntuplets"]
            out[name] = {"value": n_events * len(ms) / (sum(ms) / 1000.0), "unit": "events/s",
                         "ms_per_step": float(np.mean(ms)),
                         "efficiency": tot["matched"] / max(tot["reco"], 1),
                         "fake_rate": tot["fake"] / max(tot["nt"], 1),
                         "duplicate_rate": tot["dup"] / max(tot["reco"], 1),
                         "candidates": int(n_cand), "n_ntuplets": tot["nt"]}
    return out


def _vertexing(ctx, dbat, stream, steps: int) -> dict:
    """Primary vertices (pt_find_vertices, quadruplets and longer, 0.02 cm steps) timed
    with CUDA events on the library's stream, the chain itself before the events: on 64
    PU200 events with vertex structure (200 interactions of 50 particles sharing one z,
    seeds 7300+i), and on the benchmark batch itself, whose particles each draw their own
    z0 so that the 0.02 cm linking chains thousands of tracks into a few groups (a stress
    case for the per-group sums)."""
    import torch
    out = {}
    evs = [sim.vertex_event(7300 + i, 200) for i in range(len(dbat[0][0]) - 1)]
    voff, *varrs = sim.concat(evs)
    dev = dbat[0][1].device
    vbat = (voff, *(torch.from_numpy(a).to(dev) for a in varrs))
    for name, (off, x, y, z, layer) in (("vertex_events", vbat), ("bench_batch", dbat[0])):
        ctx.pt_load_batch(off, x, y, z, layer)
        ctx.pt_build_doublets(sync=False)
        ctx.pt_connect_cells(sync=False)
        ctx.pt_find_ntuplets(sync=False)
        ctx.pt_fit_tracks(sync=False)
        nv = ctx.pt_find_vertices()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for e0, e1 in ev:
            e0.record(stream)
            ctx.pt_find_vertices(sync=False)
            e1.record(stream)
        stream.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        E = len(off) - 1
        out[name] = {"ms_per_step": statistics.mean(ms), "events_per_step": E,
                     "vertices_per_event": nv / E,
                     "tracks_per_event": ctx.pt_get_tracks().shape[0] / E}
    out["ms_per_step"] = out["vertex_events"]["ms_per_step"]
    out["workload"] = ("64 PU200 events of 200 interactions x 50 particles sharing z "
                       "(seeds 7300+i); bench_batch: the benchmark's own batch")
    return out


def _broken_line(ctx, dbat, stream, steps: int) -> dict:
    """Broken-line refit (pt_refit_broken_line, 2 % X0 per layer) of the fitted tracks of
    one bench batch, timed with CUDA events on the library's stream; the circle + line
    fit that serves as its reference runs again before each timed call, outside the
    events."""
    import torch
    off, x, y, z, layer = dbat[0]
    ctx.pt_load_batch(off, x, y, z, layer)
    ctx.pt_build_doublets(sync=False)
    ctx.pt_connect_cells(sync=False)
    ctx.pt_find_ntuplets(sync=False)
    n = ctx.pt_fit_tracks()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for e0, e1 in ev:
        ctx.pt_fit_tracks(sync=False)
        e0.record(stream)
        ctx.pt_refit_broken_line(0.02, 0.02, sync=False)
        e1.record(stream)
    stream.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    E = len(off) - 1
    return {"ms_per_step": statistics.mean(ms), "events_per_step": E, "tracks_per_step": n,
            "tracks_per_s": n / (statistics.mean(ms) / 1000.0),
            "workload": "the bench batch's fitted tracks, refitted with 2 % X0 per layer"}


def _raw_input(ctx, dev, stream, steps: int, B: int) -> dict:
    """Raw pixel data -> hits (pt_load_raw: unpack, cluster, place, bin) on B copies of
    one PU200 event's digis in device memory, timed with CUDA events on the library's
    stream (the call's host checks and the copy of the digis into the library's
    scratch included)."""
    import torch
    from sim import pixels
    words = pixels.digitize(make_events(1, SEED0 + 900)[0])[0]
    off, allw = pixels.concat_raw([words] * B)
    dw = torch.from_numpy(allw.view(np.int64)).to(dev)
    ctx.pt_set_modules()
    nh = ctx.pt_load_raw(off, dw)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        ctx.pt_load_raw(off, dw, sync=False)
        e1.record(stream)
    stream.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"ms_per_step": statistics.mean(ms), "events_per_step": B,
            "digis_per_event": int(words.size), "hits_per_event": nh / B,
            "workload": "one PU200 event's digis, repeated"}


def _physics(ctx, host, events):
    """Efficiency, fake and duplicate rates of the cleaned ntuplets (generator truth)."""
    from sim import truth
    tot = dict(reco=0, matched=0.0, fake=0, nt=0, dup=0.0)
    for bi, h in enumerate(host):
        hits, nh, tr, eoff = ctx.pt_reconstruct_batch(*h)
        for e in range(len(eoff) - 1):
            ev = events[bi * (len(eoff) - 1) + e]
            r = truth.rates_fast(hits[eoff[e]:eoff[e + 1]], ev.pid, ev.layer)
            tot["reco"] += r["n_reconstructable"]
            tot["matched"] += r["efficiency"] * r["n_reconstructable"]
            tot["dup"] += r["duplicate_rate"] * r["n_reconstructable"]
            tot["fake"] += r["n_fake"]
            tot["nt"] += r["n_ntuplets"]
    return {"efficiency": tot["matched"] / max(tot["reco"], 1),
            "fake_rate": tot["fake"] / max(tot["nt"], 1),
            "duplicate_rate": tot["dup"] / max(tot["reco"], 1),
            "n_fake": tot["fake"], "n_ntuplets": tot["nt"], "events": len(events)}


def _serving(pt, rates, seconds: float, gate=None, threads: int = 16,
             budget: int = 2 << 30, slots: int = 4, instances: int = 1) -> list:
    """Open-loop Poisson arrivals of PU 50-200 events from `threads` native client threads
    (lib/serve_load: each client submits at its arrival times and never waits for its
    results; a collector thread per client polls them) into a pt_server with a
    `budget`-byte device budget, at each offered rate in `rates`.  Per rate: completions
    over the offered window (sustained events/s), the server's latency percentiles
    (submit to result ready) and the clients' (submit to poll returning)."""
    from paper_2501_05520_gb300 import build as pbuild
    pus = sim.serving_pileups(6000, 96, 50, 200)
    pool = [sim.pileup_event(6000 + i, int(pu)) for i, pu in enumerate(pus)]
    with tempfile.TemporaryDirectory() as td:
        evf = os.path.join(td, "events.bin")
        with open(evf, "wb") as f:
            for e in pool:
                f.write(np.int64(e.n_hits).tobytes())
                for a in (e.x, e.y, e.z):
                    f.write(np.ascontiguousarray(a, "<f4").tobytes())
                f.write(np.ascontiguousarray(e.layer, np.uint8).tobytes())
        gf = "-"
        if gate is not None:
            gf = os.path.join(td, "gate.bin")
            np.concatenate([gate[0].astype("<f4"), np.array([gate[1]], "<f4")]).tofile(gf)
        c = pt.default_cuts()
        env = dict(os.environ, PT_CUTS=",".join(repr(float(np.float32(c[k]))) for k in
                                                ("kmax", "z0max", "cotmax", "rz0", "rz1",
                                                 "dca_b0", "dca_other")))
        out = []
        for rate in rates:
            r = subprocess.run([pbuild.SERVE_LOAD, evf, str(rate), str(seconds), str(threads),
                                str(slots), str(budget), gf, "11", str(instances)],
                               capture_output=True,
                               text=True, env=env, timeout=600)
            if r.returncode != 0:
                raise RuntimeError(f"serve_load failed: {r.stderr.strip()[-300:]}")
            d = json.loads(r.stdout.strip().splitlines()[-1])
            d["p50_ms"], d["p99_ms"] = d["server_p50_ms"], d["server_p99_ms"]
            d["budget_bytes"] = budget
            d["workload"] = "PU uniform in [50, 200], 50 particles per unit, 2% noise"
            out.append(d)
    return out


def run_ours(args):
    import torch
    import paper_2501_05520_gb300 as pt
    rank, world, local = _dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B = args.batch
    events = make_events(2 * B, seed0=rank_seed0(rank))
    host = [sim.concat(events[:B]), sim.concat(events[B:])]
    dbat = [(h[0], *(torch.from_numpy(a).to(dev) for a in h[1:])) for h in host]
    stream = torch.cuda.Stream(dev)
    # azimuthal bins and launch sizes: measured on this batch unless all three are given
    launch = dict(phi_bins=args.phi_bins, blocks_per_sm=args.blocks_per_sm,
                  search_blocks_per_sm=args.search_blocks_per_sm, source="command line")
    if not all(launch[k] for k in ("phi_bins", "blocks_per_sm", "search_blocks_per_sm")):
        from paper_2501_05520_gb300 import autotune
        t = autotune.tuned(*host[0], capacity(B), device=local)
        launch = {k: args.__dict__[k] or t[k]
                  for k in ("phi_bins", "blocks_per_sm", "search_blocks_per_sm")}
        launch.update(source=f"autotuned ({t['source']})", table=t["table"])
    ctx = pt.Context(capacity=capacity(B, launch["phi_bins"]), device=local, stream=stream)
    ctx.pt_set_launch(launch["blocks_per_sm"], launch["search_blocks_per_sm"])
    # the end-to-end leg's further host threads, each with a context and stream of its own
    e2e_more = [pt.Context(capacity=capacity(B, launch["phi_bins"]), device=local,
                           stream=torch.cuda.Stream(dev)) for _ in range(E2E_THREADS - 1)]
    for c in e2e_more:
        c.pt_set_launch(launch["blocks_per_sm"], launch["search_blocks_per_sm"])
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    gw, gtau = pt.default_gate()
    forms = {}
    counts = None
    clocks = None
    kernels, launches = {}, {}
    for form in ("plain", "gated"):
        ctx.pt_set_gate(gw if form == "gated" else None, gtau)
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                off, x, y, z, layer = dbat[i % 2]
                ctx.pt_enqueue_batch(off, x, y, z, layer)
            stream.synchronize()
            ctx.pt_get_ntuplets()  # raises on any capacity or input error
            if form == "plain":
                off, x, y, z, layer = dbat[0]
                ctx.pt_load_batch(off, x, y, z, layer)
                counts = dict(hits=int(off[-1]), cells=ctx.pt_build_doublets(),
                              links=ctx.pt_connect_cells(), survivors=ctx.pt_find_ntuplets())
                _, cnh, _, _ = ctx.pt_get_candidates()
                counts["candidates"] = int(cnh.size)
                counts["incidences"] = int(cnh.astype(np.int64).sum() - cnh.size)
                counts["survivor_hits"] = int(ctx.pt_get_ntuplets()[1].astype(np.int64).sum())
                ctx.pt_fit_tracks()
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            if form == "plain":
                with Clocks(local) as clk:
                    step_ms, stage_ms = _timed(ctx, dbat, args.steps, flush, stream)
                clocks = clk.summary()
            else:
                step_ms, stage_ms = _timed(ctx, dbat, args.steps, flush, stream)
            torch.cuda.synchronize(dev)
            if dist:
                dist.barrier()
            ctx.pt_get_ntuplets()
            # per-kernel device times, on extra steps after the timed region
            ctx.pt_set_tracing(True)
            _timed(ctx, dbat, TRACE_STEPS, flush, stream)
            trace = ctx.pt_get_trace()
            ctx.pt_set_tracing(False)
            kernels[form] = {k: round(ms / n, 4) for k, (ms, n) in trace.items()}
            launches[form] = sum(n * (3 if k == "scan" else 1)
                                 for k, (_, n) in trace.items()) // TRACE_STEPS
        total_s = max_over_ranks(sum(step_ms) / 1000.0, dist, dev)
        # end to end through the public call: pinned host in, host out; E2E_THREADS host
        # threads, each with its own context and stream, so one batch's copies overlap the
        # others' kernels
        e2e_s, S = 0.0, 0
        if not args.no_e2e:
            for c in e2e_more:
                c.pt_set_gate(gw if form == "gated" else None, gtau)
            e2e_s, S = _e2e(pt, [ctx] + e2e_more, host[0], B, args.steps, args.warmup)
        e2e_s = max_over_ranks(e2e_s, dist, dev)
        forms[form] = dict(
            value=job_rate(world, B, args.steps, total_s), ms_per_step=1000.0 * total_s / args.steps,
            p99_ms_per_step=float(np.percentile(step_ms, 99)),
            stages_ms={n: round(statistics.mean(v), 4) for n, v in stage_ms.items()},
            e2e=None if args.no_e2e else {
                 "value": job_rate(world, B, args.steps, e2e_s), "unit": "events/s",
                 "host_threads": E2E_THREADS,
                 "h2d_bytes_per_step": int(host[0][0][-1]) * 13 + (B + 1) * 4 + 8,
                 "d2h_bytes_per_step": S * (24 + 1 + 36) + (B + 1) * 8 + 128},
            physics=_physics(ctx, host, events) if not args.no_physics else None)
    ctx.pt_set_gate(None, 0.0)
    with torch.cuda.stream(stream):
        vertexing = _vertexing(ctx, dbat, stream, min(args.steps, 20))
        broken_line = _broken_line(ctx, dbat, stream, min(args.steps, 20))
        raw_input = _raw_input(ctx, dev, stream, min(args.steps, 20), B)
    latency = _latency(pt, dev) if not args.no_latency else None
    gap = _gap_form(pt, dev, flush, min(args.steps, 10)) if not args.no_physics else None
    fishbone = _fishbone_form(pt, dev, flush, min(args.steps, 10)) if not args.no_physics else None
    config4 = {"plain": _config4(ctx, dev, flush, stream, args.steps, args.warmup, B)}
    ctx.pt_set_gate(gw, gtau)
    config4["gated"] = _config4(ctx, dev, flush, stream, args.steps, args.warmup, B)
    ctx.pt_set_gate(None, 0.0)

    # roofline of the dominant kernel of the plain form: its step's algorithmic bytes over
    # the kernel's mean traced launch time; the same bytes over the whole step call's time,
    # and every step of the chain, beside it
    plain = forms["plain"]
    km = kernels["plain"]
    peaks = _peaks()
    pk = peaks["hbm_gbs"]
    dom = max((k for k in km if k in KERNEL_STAGE), key=lambda k: km[k])
    dstage = KERNEL_STAGE[dom]
    ab = stage_bytes(dstage, counts)
    achieved = ab / (km[dom] / 1000.0) / 1e9
    rec = NCU_TRAFFIC.get(dom)
    fresh = rec is not None and rec["sha"] == kernel_sources_sha(dom)
    traffic = int(rec["bytes_per_event"] * B) if fresh else None
    steps_frac = {}
    for call, st in CALL_STAGES.items():
        by = sum(stage_bytes(x, counts) for x in st)
        ms = plain["stages_ms"][call]
        steps_frac["+".join(st)] = {"bytes": by, "ms": ms,
                                    "achieved_gbs": round(by / (ms / 1000.0) / 1e9, 1),
                                    "frac": round(by / (ms / 1000.0) / 1e9 / pk, 4)}
    graph = [c for c in CALL_STAGES if c != "fit"]
    gby = sum(steps_frac["+".join(CALL_STAGES[c])]["bytes"] for c in graph)
    gms = sum(plain["stages_ms"][c] for c in graph)
    call_of = {st[0]: c for c, st in CALL_STAGES.items()}
    sms_ = plain["stages_ms"][call_of[dstage]] if dstage in call_of else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved,
                "peak": pk, "unit": "GB/s", "frac": achieved / pk,
                "traffic": traffic, "peak_src": peaks["src"],
                "algorithmic_bytes": ab, "bytes_source": f"step {dstage} accounting",
                "launch_ms": km[dom],
                "traffic_over_algorithmic": round(traffic / ab, 3) if traffic else None,
                "layout_bytes": kernel_layout_bytes(dom, counts),
                "issue_active_pct": rec["issue_active_pct"] if fresh else None,
                "issue": _issue_roof(rec if fresh else None, B, km[dom], clocks),
                "stage": {"name": dstage, "ms": sms_,
                          "frac": round(ab / (sms_ / 1000.0) / 1e9 / pk, 4) if sms_ else None},
                "graph_stages_A1_A6": {"bytes": gby, "ms": round(gms, 4),
                                       "frac": round(gby / (gms / 1000.0) / 1e9 / pk, 4)},
                "steps": steps_frac}

    if rank == 0:
        line = {"metric": METRIC, "value": plain["value"], "unit": "events/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": plain["ms_per_step"], "p99_ms_per_step": plain["p99_ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "events_per_step": B, "form": "plain",
                           "phi_bins": launch["phi_bins"],
                           "blocks_per_sm": launch["blocks_per_sm"],
                           "search_blocks_per_sm": launch["search_blocks_per_sm"],
                           "tuning": launch["source"],
                           "l2": "flushed before every step (256 MB write, outside the events)",
                           "parallelism": f"replicas x{world}"},
                "e2e": plain["e2e"],
                "roofline": roofline,
                "stages_ms": plain["stages_ms"],
                "kernels_ms": kernels["plain"],
                "gated": dict({k: forms["gated"][k] for k in ("value", "ms_per_step",
                                                              "p99_ms_per_step", "stages_ms",
                                                              "e2e")},
                              kernels_ms=kernels["gated"]),
                "physics": {"plain": plain["physics"], "gated": forms["gated"]["physics"]},
                "counts_per_step": counts,
                "batch_workload": config4,
                "latency": latency,
                "gap_pairs": gap,
                "fishbone": fishbone,
                "vertexing": vertexing,
                "broken_line": broken_line,
                "raw_input": raw_input,
                "autotune": launch,
                "clocks": clocks,
                "gpu_launches": launches["plain"] * args.steps}
        if not args.no_serving:
            rates = [float(r) for r in args.serve_rates.split(",")]
            line["serving"] = {
                form: _serving(pt, rates, args.serve_seconds,
                               gate=(gw, gtau) if form == "gated" else None)
                for form in ("plain", "gated")}
            # model-instance scaling on one GPU: 1, 2 and 4 server instances behind the
            # router, offered more than one instance sustains
            line["serving"]["instances"] = [
                _serving(pt, [args.serve_instances_rate], args.serve_seconds, instances=k)[0]
                for k in (1, 2, 4)]
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    ctx.close()
    for c in e2e_more:
        c.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--phi-bins", type=int, default=0, help="0: autotuned")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="0: autotuned")
    ap.add_argument("--search-blocks-per-sm", type=int, default=0, help="0: autotuned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-physics", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer rate (profiling)")
    ap.add_argument("--no-latency", action="store_true", help="skip the single-event latencies")
    ap.add_argument("--serve-rates", default="200,1000,2000,4000,6000,8000,10000,12000",
                    help="offered events/s of the serving sweep")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-instances-rate", type=float, default=16000.0,
                    help="offered events/s of the instance-scaling runs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        import paper_2501_05520_gb300.build as b
        b.build()
        run_ours(args)


if __name__ == "__main__":
    main()
