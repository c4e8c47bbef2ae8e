"""Request server (continuous batching): every result equals the event run alone, under
concurrent submission from many threads with mixed event sizes; poll semantics,
admission errors, statistics, and the gated form."""

import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import sim
from parity import assert_fits_close, assert_ntuplets_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

ALONE_CAP = pt.default_capacity(max_events=1, hits_per_event=65536, cells_per_event=4 << 20,
                                links_per_event=1 << 20, ntuplets_per_event=1 << 19)


def _events(n, seed0):
    pus = sim.serving_pileups(seed0, n, lo=20, hi=200)
    return [sim.pileup_event(seed0 + i, int(pu)) for i, pu in enumerate(pus)]


def _alone(events, cuts, gate=None):
    out = []
    with pt.Context(cuts=cuts, capacity=ALONE_CAP) as ctx:
        if gate is not None:
            ctx.pt_set_gate(*gate)
        for ev in events:
            h, n, t, _ = ctx.pt_reconstruct_batch([0, ev.n_hits], ev.x, ev.y, ev.z, ev.layer)
            out.append((h.copy(), n.copy(), t.copy()))
    return out


def _serve(server, events, threads=8):
    def one(ev):
        t = server.pt_submit(ev.x, ev.y, ev.z, ev.layer)
        return server.pt_poll(t, timeout_us=-1)
    with cf.ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, events))


def test_results_same_alone_and_in_the_mix(cuts):
    events = _events(40, 6000)
    ref = _alone(events, cuts)
    with pt.Server(cuts=cuts, budget_bytes=3 << 30, slots=3) as srv:
        got = _serve(srv, events, threads=16)
        st = srv.pt_server_stats()
    for (h, n, t), (h2, n2, t2) in zip(ref, got):
        assert np.array_equal(h, h2) and np.array_equal(n, n2)
        assert t.tobytes() == t2.tobytes()
    assert st["n_done"] == len(events)
    assert 0 < st["p50_ms"] <= st["p99_ms"] and st["events_per_s"] > 0
    # served results against the oracle directly, on a sample of the mix
    for i in (0, 7, 19, 33):
        ev = events[i]
        ref_o = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        h, n, t = got[i]
        assert_ntuplets_equal(h, oracle.survivors_hits(ref_o), ref_o)
        assert_fits_close(t, ref_o["fit"])


def test_gated_serving_same_as_gated_alone(cuts):
    events = _events(12, 6100)
    gate = pt.default_gate()
    ref = _alone(events, cuts, gate=gate)
    with pt.Server(cuts=cuts, budget_bytes=2 << 30, slots=2) as srv:
        srv.pt_server_set_gate(*gate)
        got = _serve(srv, events)
    for (h, n, t), (h2, n2, t2) in zip(ref, got):
        assert np.array_equal(h, h2) and t.tobytes() == t2.tobytes()


def test_poll_admission_and_errors(cuts):
    with pt.Server(cuts=cuts, budget_bytes=1 << 30, slots=1) as srv:
        with pytest.raises(pt.PtError) as ei:
            srv.pt_poll(12345, 0)
        assert ei.value.status == pt.PT_ERR_INVALID
        big = sim.pileup_event(6200, 400)
        assert big.n_hits > 65536
        with pytest.raises(pt.PtError) as ei:
            srv.pt_submit(big.x, big.y, big.z, big.layer)
        assert ei.value.status == pt.PT_ERR_CAPACITY
        bad = sim.pileup_event(6201, 10)
        layer = bad.layer.copy()
        layer[0] = 12
        with pytest.raises(pt.PtError) as ei:
            srv.pt_submit(bad.x, bad.y, bad.z, layer)
        assert ei.value.status == pt.PT_ERR_INVALID
        ev = sim.pileup_event(6202, 200)
        t = srv.pt_submit(ev.x, ev.y, ev.z, ev.layer)
        try:
            srv.pt_poll(t, timeout_us=1)
        except pt.PtError as e:
            assert e.status in (pt.PT_ERR_TIMEOUT, pt.PT_ERR_NOT_READY)
            h, n, tr = srv.pt_poll(t, timeout_us=5_000_000)
            assert h.shape[0] > 1000
        # the ticket is released after a successful poll
        with pytest.raises(pt.PtError):
            srv.pt_poll(t, 0)


def test_native_load_generator(cuts, tmp_path):
    """lib/serve_load (native client threads, open-loop arrivals): every submitted event
    completes without error and the server's statistics count them all."""
    import json
    import os
    import subprocess
    from paper_2501_05520_gb300 import build as pbuild
    pool = _events(12, 6100)
    evf = tmp_path / "events.bin"
    with open(evf, "wb") as f:
        for e in pool:
            f.write(np.int64(e.n_hits).tobytes())
            for a in (e.x, e.y, e.z):
                f.write(np.ascontiguousarray(a, "<f4").tobytes())
            f.write(np.ascontiguousarray(e.layer, np.uint8).tobytes())
    env = dict(os.environ, PT_CUTS=",".join(repr(float(np.float32(cuts[k]))) for k in
                                            ("kmax", "z0max", "cotmax", "rz0", "rz1", "dca_b0",
                                             "dca_other")))
    r = subprocess.run([pbuild.SERVE_LOAD, str(evf), "300", "0.5", "4", "2", str(2 << 30), "-",
                        "3"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["errors"] == 0 and d["submitted"] > 50 and d["completed"] == d["submitted"]
    assert 0 < d["server_p50_ms"] <= d["server_p99_ms"]


def test_router_results_same_alone(cuts):
    """Three server instances behind the router: every result equals the event alone,
    and the requests spread over the instances."""
    events = _events(30, 6200)
    ref = _alone(events, cuts)
    with pt.Router(instances=3, cuts=cuts, budget_bytes_per_instance=1 << 30, slots=2) as r:
        got = _serve(r, events, threads=12)
        st = r.pt_server_stats()
    for (h, n, t), (h2, n2, t2) in zip(ref, got):
        assert np.array_equal(h, h2) and np.array_equal(n, n2)
        assert t.tobytes() == t2.tobytes()
    assert st["n_done"] == len(events) and sum(st["per_instance"]) == len(events)
    assert sum(1 for k in st["per_instance"] if k > 0) >= 2
