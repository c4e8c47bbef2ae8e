"""Host logic of the N-replica benchmark on two gloo ranks (CPU): every rank draws its own
event stream, the job time is the slowest rank's, the rate counts every rank's events,
and the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 0.5 + rank  # rank 1 is the slow one
        t = bench.max_over_ranks(mine, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed0(rank))
        q.put((rank, t, seeds, bench.job_rate(world, 64, 10, t), bench._dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, seeds, rate, env in out:
        assert t == 1.5                       # max over ranks, on every rank
        assert rate == 2 * 64 * 10 / 1.5      # both ranks' events over the slowest time
        assert env == (rank, 2, rank)
        # disjoint seed ranges: each rank draws 2 x batch events from its first seed
        assert seeds[1] - seeds[0] >= 2 * bench.BATCH
    assert bench.max_over_ranks(0.25) == 0.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(a))

    class A:
        steps, warmup = 2, 3
    bench.run_reference(A())
    assert called == [] and capsys.readouterr().out == ""


def test_reference_arm_json_line(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the contract's keys; the oracle's timing is
    stubbed (4 events at 2 events/s per call)."""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "cpu_baseline",
                        lambda n, **k: {"value": 2.0, "unit": "events/s", "cores": n,
                                        "kind": "oracle", "sample": "stub"})

    class A:
        steps, warmup, gpus = 3, 3, 1
    bench.run_reference(A())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] == pytest.approx(2.0) and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
