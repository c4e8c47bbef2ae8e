"""pt_find_doublets_noalloc: the allocation-free doublet search for callers that cannot
allocate device memory, checked against the oracle and the context-based entry point.

Two calls in a row on different events: each call must return exactly the oracle's
doublet set for the same event and cuts, which is also what pt_build_doublets +
pt_get_cells return (integer output, so the comparison is exact).  The calls go
through the C ABI with device buffers the test owns; the function itself allocates
nothing.
"""

import ctypes

import numpy as np
import pytest

import oracle
import sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402

CAP = pt.default_capacity(max_events=1, hits_per_event=65536, cells_per_event=4 << 20,
                          links_per_event=1 << 20, ntuplets_per_event=1 << 19)


class _Hits:
    """Bare hit arrays with the attributes _noalloc reads."""

    def __init__(self, x, y, z, layer):
        self.x, self.y, self.z, self.layer = x, y, z, layer
        self.n_hits = int(x.shape[0])


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
        ref = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
        assert got == set(zip(ref["cell_inner"].tolist(), ref["cell_outer"].tolist()))


def test_noalloc_limits(cuts):
    ev = sim.generate(sim.PU50, 2061)
    st, n, _, _ = _noalloc(ev, cuts, 100)
    assert st == pt.PT_ERR_CAPACITY and n > 100
    big = sim.generate(sim.PU200, 3071, n_particles=16000)
    assert big.n_hits > 65536
    st, _, _, _ = _noalloc(big, cuts, 16)
    assert st == pt.PT_ERR_CAPACITY
    assert "65536" in pt.lib().pt_last_error().decode()


def test_noalloc_edge_cases(cuts):
    """An empty event gives no doublets; a layer code of 10 is refused; a second call
    leaves the device's free memory unchanged (the call allocates nothing)."""
    ev = sim.generate(sim.PU50, 2062)
    empty = _Hits(ev.x[:0], ev.y[:0], ev.z[:0], ev.layer[:0])
    st, n, _, _ = _noalloc(empty, cuts, 16)
    assert st == pt.PT_OK and n == 0
    layer = ev.layer.copy()
    layer[17] = 10
    st, _, _, _ = _noalloc(_Hits(ev.x, ev.y, ev.z, layer), cuts, 4 << 20)
    assert st == pt.PT_ERR_INVALID
    st, n1, _, _ = _noalloc(ev, cuts, 4 << 20)
    assert st == pt.PT_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st, n2, _, _ = _noalloc(ev, cuts, 4 << 20)
    torch.cuda.synchronize()
    assert st == pt.PT_OK and n2 == n1
    assert torch.cuda.mem_get_info()[0] == free0
