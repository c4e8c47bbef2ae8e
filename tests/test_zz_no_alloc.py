"""pt_find_doublets_noalloc: the allocation-free doublet search for callers that cannot
allocate device memory, checked against the context-based entry point.

Two calls in a row on different events: each call must return exactly the doublet set
that pt_build_doublets + pt_get_cells returns for the same event and cuts (integer
output, so the comparison is exact).  The calls go through the C ABI with device
buffers the test owns; the function itself allocates nothing.
"""

import ctypes

import numpy as np
import pytest

import sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

CAP = pt.default_capacity(max_events=1, hits_per_event=65536, cells_per_event=4 << 20,
                          links_per_event=1 << 20, ntuplets_per_event=1 << 19)


def _noalloc(ev, cuts, cap):
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ev.x, ev.y, ev.z, ev.layer)]
    inner = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    outer = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    c = pt.PtCuts(*(float(cuts[k]) for k, _ in pt.PtCuts._fields_))
    stream = torch.cuda.current_stream().cuda_stream
    st = pt.lib().pt_find_doublets_noalloc(
        ctypes.byref(c), ev.n_hits, *(ctypes.c_void_p(t.data_ptr()) for t in dev),
        ctypes.c_void_p(inner.data_ptr()), ctypes.c_void_p(outer.data_ptr()), cap,
        ctypes.byref(n), ctypes.c_void_p(stream) if stream else None)
    return st, int(n.value), inner.cpu().numpy(), outer.cpu().numpy()


def _reference(ev, cuts):
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
        ctx.pt_build_doublets()
        a, b, _ = ctx.pt_get_cells()
    return set(zip(a.tolist(), b.tolist()))


def test_noalloc_doublets_match_context_entry_point(cuts):
    for ev in (sim.generate(sim.PU50, 2060), sim.generate(sim.PU200, 3070)):
        exp = _reference(ev, cuts)
        st, n, inner, outer = _noalloc(ev, cuts, 4 << 20)
        assert st == pt.PT_OK, pt.lib().pt_last_error().decode()
        assert n == len(exp)
        got = set(zip(inner[:n].tolist(), outer[:n].tolist()))
        assert len(got) == n and got == exp


def test_noalloc_limits(cuts):
    ev = sim.generate(sim.PU50, 2061)
    st, n, _, _ = _noalloc(ev, cuts, 100)
    assert st == pt.PT_ERR_CAPACITY and n > 100
    big = sim.generate(sim.PU200, 3071, n_particles=16000)
    assert big.n_hits > 65536
    st, _, _, _ = _noalloc(big, cuts, 16)
    assert st == pt.PT_ERR_CAPACITY
    assert "65536" in pt.lib().pt_last_error().decode()
