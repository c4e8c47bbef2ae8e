"""GB300 pixel-track cellular automaton: thin Python binding of the C ABI in include/pt_ca.h.

Argument marshalling only: every stage of the chain runs in the CUDA library
(lib/libptca.so).  There is no CPU fallback: if the library is missing, every call
raises.  PyTorch is used only for device memory (the workspace) and the stream.

Function names follow the C ABI (pt_create, pt_load_hits, pt_build_doublets, ...);
`Context` bundles a context handle with its torch-allocated workspace.
"""

from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# PT_DEBUG=1 in the environment selects the debug build (bounds-checked kernels,
# build.build(debug=True)).
LIB_PATH = os.path.join(_PKG, "lib", "libptca_debug.so" if os.environ.get("PT_DEBUG") == "1"
                        else "libptca.so")
CUTS_FILE = os.path.join(_PKG, "params", "cuts_v1.json")
_lib = None

PT_OK, PT_ERR_INVALID, PT_ERR_CAPACITY, PT_ERR_CUDA, PT_ERR_TIMEOUT, PT_ERR_NOT_READY, \
    PT_ERR_NOMEM, PT_ERR_INTERNAL = range(8)

# Every symbol include/pt_ca.h declares.
EXPORTED = ("pt_workspace_size", "pt_create", "pt_destroy", "pt_set_stream", "pt_load_hits",
            "pt_load_batch", "pt_build_doublets", "pt_connect_cells", "pt_find_ntuplets",
            "pt_fit_tracks", "pt_refit_broken_line", "pt_get_ntuplets", "pt_get_tracks",
            "pt_find_vertices",
            "pt_set_modules", "pt_load_raw", "pt_get_hits",
            "pt_get_vertices", "pt_get_cells", "pt_get_links",
            "pt_get_candidates", "pt_reconstruct_batch", "pt_enqueue_batch",
            "pt_find_doublets_noalloc", "pt_set_gate", "pt_get_link_features", "pt_gate_score",
            "pt_gate_loss_grad", "pt_gate_adam", "pt_server_create", "pt_server_set_gate",
            "pt_submit", "pt_poll", "pt_server_stats", "pt_server_reset_stats",
            "pt_server_destroy", "pt_set_launch", "pt_autotune", "pt_set_tracing",
            "pt_get_trace", "pt_set_layer_pairs", "pt_set_wait_limit", "pt_set_fishbone", "pt_debug_build",
            "pt_debug_inject",
            "pt_server_counters",
            "pt_router_create", "pt_router_set_gate", "pt_router_submit", "pt_router_poll",
            "pt_router_stats", "pt_router_reset_stats", "pt_router_destroy", "pt_last_error")


# The chain's 13 (inner, outer) layer pairs, the library's default table (pt_set_layer_pairs).
DEFAULT_PAIRS = ((0, 1), (1, 2), (2, 3), (0, 4), (1, 4), (2, 4), (4, 5), (5, 6),
                 (0, 7), (1, 7), (2, 7), (7, 8), (8, 9))


def gap_pairs(pairs=DEFAULT_PAIRS) -> tuple:
    """Skip-layer pairs of a table: (a, c) for each a -> b -> c of its pair graph that is
    not itself a pair, so a track that misses layer b still joins a and c."""
    have = set(pairs)
    return tuple(sorted({(a, c) for a, b in pairs for b2, c in pairs
                         if b2 == b and (a, c) not in have}))


class PtCuts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_float), ("z0max", ctypes.c_float), ("cotmax", ctypes.c_float),
                ("rz0", ctypes.c_float), ("rz1", ctypes.c_float), ("dca_b0", ctypes.c_float),
                ("dca_other", ctypes.c_float)]


class PtKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("total_ms", ctypes.c_double),
                ("launches", ctypes.c_int64)]


class PtGeometry(ctypes.Structure):
    _fields_ = [("bfield_T", ctypes.c_float)]


class PtCapacity(ctypes.Structure):
    _fields_ = [("max_events", ctypes.c_int64), ("max_hits", ctypes.c_int64),
                ("max_cells", ctypes.c_int64), ("max_links", ctypes.c_int64),
                ("max_ntuplets", ctypes.c_int64), ("phi_bins", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


TRACK_DTYPE = np.dtype([("kappa", "<f4"), ("phi0", "<f4"), ("d0", "<f4"), ("cot_theta", "<f4"),
                        ("z0", "<f4"), ("pt", "<f4"), ("chi2_circle", "<f4"),
                        ("chi2_line", "<f4"), ("charge", "i1"), ("nhits", "u1"),
                        ("pad", "u1", (2,))])
assert TRACK_DTYPE.itemsize == 36
VERTEX_DTYPE = np.dtype([("z", "<f4"), ("sum_pt2", "<f4"), ("n_tracks", "<i4"), ("event", "<i4")])
assert VERTEX_DTYPE.itemsize == 16


class PtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pt status {status}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2501_05520_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        PI64 = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "pt_workspace_size": [ctypes.POINTER(PtCapacity), ctypes.POINTER(ctypes.c_size_t)],
            "pt_create": [ctypes.POINTER(PtGeometry), ctypes.POINTER(PtCuts),
                          ctypes.POINTER(PtCapacity), I32, P, ctypes.c_size_t, P,
                          ctypes.POINTER(ctypes.c_void_p)],
            "pt_destroy": [P],
            "pt_set_stream": [P, P],
            "pt_load_hits": [P, I64, P, P, P, P, I32],
            "pt_load_batch": [P, I32, P, P, P, P, P, I32],
            "pt_build_doublets": [P, PI64],
            "pt_connect_cells": [P, PI64],
            "pt_find_ntuplets": [P, PI64],
            "pt_fit_tracks": [P, PI64],
            "pt_refit_broken_line": [P, ctypes.c_float, ctypes.c_float, PI64],
            "pt_get_ntuplets": [P, P, P, P, I64, PI64, I32],
            "pt_get_tracks": [P, P, I64, PI64, I32],
            "pt_find_vertices": [P, I32, ctypes.c_float, PI64],
            "pt_set_modules": [P, P, I32],
            "pt_load_raw": [P, I32, P, P, I32, PI64],
            "pt_get_hits": [P, P, P, P, P, P, I64, PI64],
            "pt_get_vertices": [P, P, P, P, I64, PI64, I32],
            "pt_get_cells": [P, P, P, P, I64, PI64],
            "pt_get_links": [P, P, P, P, P, P, I64, PI64],
            "pt_get_candidates": [P, P, P, P, P, I64, PI64],
            "pt_reconstruct_batch": [P, I32, P, P, P, P, P, I32, P, P, P, P, I64, PI64, I32],
            "pt_enqueue_batch": [P, I32, P, P, P, P, P, I32],
            "pt_find_doublets_noalloc": [ctypes.POINTER(PtCuts), I64, P, P, P, P, P, P, I64,
                                         PI64, P],
            "pt_set_gate": [P, P, ctypes.c_float],
            "pt_get_link_features": [P, P, P, P, P, P, P, I64, PI64],
            "pt_gate_score": [P, P, I64, P],
            "pt_gate_loss_grad": [P, P, P, I64, P, P, P],
            "pt_gate_adam": [P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, I32, P],
            "pt_server_create": [ctypes.POINTER(PtGeometry), ctypes.POINTER(PtCuts), I32,
                                 ctypes.c_size_t, I32, ctypes.POINTER(ctypes.c_void_p)],
            "pt_server_set_gate": [P, P, ctypes.c_float],
            "pt_submit": [P, I64, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)],
            "pt_poll": [P, ctypes.c_uint64, I64, P, P, P, I64, PI64],
            "pt_server_stats": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), PI64],
            "pt_server_reset_stats": [P],
            "pt_server_counters": [P, PI64, PI64, PI64],
            "pt_router_create": [ctypes.POINTER(PtGeometry), ctypes.POINTER(PtCuts), P, I32,
                                 ctypes.c_size_t, I32, ctypes.POINTER(ctypes.c_void_p)],
            "pt_router_set_gate": [P, P, ctypes.c_float],
            "pt_router_submit": [P, I64, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)],
            "pt_router_poll": [P, ctypes.c_uint64, I64, P, P, P, I64, PI64],
            "pt_router_stats": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), PI64, P],
            "pt_router_reset_stats": [P],
            "pt_router_destroy": [P],
            "pt_server_destroy": [P],
            "pt_set_launch": [P, I32, I32],
            "pt_set_layer_pairs": [P, I32, P, P],
            "pt_set_wait_limit": [P, I64],
            "pt_set_fishbone": [P, I32],
            "pt_debug_build": [],
            "pt_debug_inject": [P, I32],
            "pt_set_tracing": [P, I32],
            "pt_get_trace": [P, P, I32, P],
            "pt_autotune": [ctypes.POINTER(PtGeometry), ctypes.POINTER(PtCuts),
                            ctypes.POINTER(PtCapacity), I32, I32, P, P, P, P, P, P, I32, P, I32,
                            P, I32, I32, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.pt_last_error.restype = ctypes.c_char_p
        L.pt_last_error.argtypes = []
        _lib = L
    return _lib


def _check(status: int):
    if status != PT_OK:
        raise PtError(status, lib().pt_last_error().decode())


def default_cuts(which: str = "pt_min_0p45") -> dict:
    """Frozen float32 cut constants (params/cuts_v1.json)."""
    with open(CUTS_FILE) as f:
        d = json.load(f)[which]
    return {k: d[k] for k, _ in PtCuts._fields_}


GATE_FILE = os.path.join(_PKG, "params", "gate_v1.npz")


def default_gate():
    """(weights float32 [5057], tau) of the trained gate shipped with the library."""
    d = np.load(GATE_FILE)
    return d["w"].astype(np.float32), float(d["tau"])


def default_capacity(max_events: int = 1, hits_per_event: int = 65536,
                     cells_per_event: int = 4 << 20, links_per_event: int = 1 << 20,
                     ntuplets_per_event: int = 1 << 19, phi_bins: int = 256) -> dict:
    return dict(max_events=max_events, max_hits=max_events * hits_per_event,
                max_cells=max_events * cells_per_event, max_links=max_events * links_per_event,
                max_ntuplets=min(max_events * ntuplets_per_event, (1 << 29) - 1),
                phi_bins=phi_bins, reserved=0)


def _cap(d: dict) -> PtCapacity:
    return PtCapacity(*(int(d.get(k, 0)) for k, _ in PtCapacity._fields_))


def pt_workspace_size(capacity: dict) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().pt_workspace_size(ctypes.byref(_cap(capacity)), ctypes.byref(n)))
    return int(n.value)


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_input(a, dtype):
    """(pointer, on_device, keep-alive) for a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        t = a.contiguous()
        # 64-bit raw words travel in an int64 tensor (same bits)
        want = {np.float32: torch.float32, np.uint8: torch.uint8, np.uint64: torch.int64}[dtype]
        if t.dtype != want:
            t = t.to(want)
        return ctypes.c_void_p(t.data_ptr()), int(t.is_cuda), t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return _hptr(arr), 0, arr


class Context:
    """A pt_ctx with a workspace borrowed from the torch caching allocator.

    cuts: dict of pt_cuts fields (default: the frozen constants); capacity: dict of
    pt_capacity fields; stream: a torch.cuda.Stream, or None for torch's current stream.
    """

    def __init__(self, cuts: dict | None = None, capacity: dict | None = None,
                 bfield: float = 3.8, device: int = 0, stream=None, torch_workspace: bool = True):
        import torch
        self.cuts = dict(cuts or default_cuts())
        self.capacity = dict(capacity or default_capacity())
        self.device = device
        L = lib()
        nbytes = pt_workspace_size(self.capacity)
        ws_ptr, ws_bytes = None, 0
        self._ws = None
        if torch_workspace:
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) // 256 * 256
            ws_bytes = nbytes
        if stream is None:
            stream = torch.cuda.current_stream(device)
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self.stream = stream
        h = ctypes.c_void_p(None)
        _check(L.pt_create(ctypes.byref(PtGeometry(bfield)),
                           ctypes.byref(PtCuts(*(float(self.cuts[k]) for k, _ in PtCuts._fields_))),
                           ctypes.byref(_cap(self.capacity)), device,
                           ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_bytes,
                           ctypes.c_void_p(sp) if sp else None, ctypes.byref(h)))
        self.handle = h
        self.n_events = 0

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().pt_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ stages
    def pt_load_hits(self, x, y, z, layer):
        px, dev, kx = _as_input(x, np.float32)
        py, _, ky = _as_input(y, np.float32)
        pz, _, kz = _as_input(z, np.float32)
        pl, _, kl = _as_input(layer, np.uint8)
        n = int(kx.shape[0]) if hasattr(kx, "shape") else len(kx)
        _check(lib().pt_load_hits(self.handle, n, px, py, pz, pl, dev))
        self.n_events = 1

    def pt_load_batch(self, offsets, x, y, z, layer):
        off = np.ascontiguousarray(offsets, np.int64)
        px, dev, kx = _as_input(x, np.float32)
        py, _, ky = _as_input(y, np.float32)
        pz, _, kz = _as_input(z, np.float32)
        pl, _, kl = _as_input(layer, np.uint8)
        _check(lib().pt_load_batch(self.handle, off.size - 1, _hptr(off), px, py, pz, pl, dev))
        self.n_events = off.size - 1

    def _stage(self, fn, sync: bool):
        if not sync:
            _check(fn(self.handle, None))
            return None
        n = ctypes.c_int64(0)
        _check(fn(self.handle, ctypes.byref(n)))
        return int(n.value)

    def pt_build_doublets(self, sync: bool = True):
        return self._stage(lib().pt_build_doublets, sync)

    def pt_connect_cells(self, sync: bool = True):
        return self._stage(lib().pt_connect_cells, sync)

    def pt_find_ntuplets(self, sync: bool = True):
        return self._stage(lib().pt_find_ntuplets, sync)

    def pt_fit_tracks(self, sync: bool = True):
        return self._stage(lib().pt_fit_tracks, sync)

    def pt_refit_broken_line(self, x0_barrel: float = 0.02, x0_disk: float = 0.02,
                             sync: bool = True):
        """Broken-line refit of the fitted tracks in place; returns their number when
        sync."""
        n = ctypes.c_int64(0)
        _check(lib().pt_refit_broken_line(self.handle, float(x0_barrel), float(x0_disk),
                                          ctypes.byref(n) if sync else None))
        return int(n.value) if sync else None

    # ----------------------------------------------------------------- results
    def pt_get_ntuplets(self):
        """(hits int32 [S,6] event-local, nhits uint8 [S], event_offsets int64 [E+1])."""
        n = ctypes.c_int64(0)
        st = lib().pt_get_ntuplets(self.handle, None, None, None, 0, ctypes.byref(n), 0)
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        S = int(n.value)
        hits = np.empty((S, 6), np.int32)
        nh = np.empty(S, np.uint8)
        off = np.empty(self.n_events + 1, np.int64)
        _check(lib().pt_get_ntuplets(self.handle, _hptr(hits), _hptr(nh), _hptr(off), S,
                                     ctypes.byref(n), 0))
        return hits, nh, off

    def pt_get_tracks(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        st = lib().pt_get_tracks(self.handle, None, 0, ctypes.byref(n), 0)
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        out = np.zeros(int(n.value), TRACK_DTYPE)
        _check(lib().pt_get_tracks(self.handle, _hptr(out), out.size, ctypes.byref(n), 0))
        return out

    def pt_set_modules(self, table=None):
        """Preload the pixel-readout module table (default: the library's detector)."""
        from . import pixels
        t = np.ascontiguousarray(pixels.module_table() if table is None else table,
                                 pixels.MODULE_DTYPE)
        _check(lib().pt_set_modules(self.handle, _hptr(t), int(t.size)))

    def pt_load_raw(self, digi_offsets, digis, sync: bool = True):
        """Load raw digis (uint64, host array or device tensor) of a batch; returns the
        number of hits made from them when sync."""
        off = np.ascontiguousarray(digi_offsets, np.int64)
        count = digis.numel() if hasattr(digis, "numel") else np.asarray(digis).size
        if off.size < 2 or off[-1] > count:
            raise ValueError("digi_offsets need n_events + 1 entries and at most len(digis) digis")
        ptr, on_dev, keep = _as_input(digis, np.uint64)
        n = ctypes.c_int64(0)
        _check(lib().pt_load_raw(self.handle, int(off.size - 1), _hptr(off), ptr, on_dev,
                                 ctypes.byref(n) if sync else None))
        self.n_events = int(off.size - 1)
        del keep
        return int(n.value) if sync else None

    def pt_get_hits(self):
        """(x, y, z float32 [N], layer uint8 [N], event_offsets int64 [E+1]) of the
        loaded batch."""
        n = ctypes.c_int64(0)
        st = lib().pt_get_hits(self.handle, None, None, None, None, None, 0, ctypes.byref(n))
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        N = int(n.value)
        x, y, z = (np.empty(N, np.float32) for _ in range(3))
        layer = np.empty(N, np.uint8)
        off = np.empty(self.n_events + 1, np.int64)
        _check(lib().pt_get_hits(self.handle, _hptr(x), _hptr(y), _hptr(z), _hptr(layer),
                                 _hptr(off), N, ctypes.byref(n)))
        return x, y, z, layer, off

    def pt_find_vertices(self, min_hits: int = 4, dz: float = 0.02, sync: bool = True):
        """Primary vertices of the fitted tracks; returns their number when sync."""
        n = ctypes.c_int64(0)
        _check(lib().pt_find_vertices(self.handle, int(min_hits), float(dz),
                                      ctypes.byref(n) if sync else None))
        return int(n.value) if sync else None

    def pt_get_vertices(self):
        """(vertices VERTEX_DTYPE [V], event_offsets int64 [E+1], track_vertex int32 [S])."""
        n = ctypes.c_int64(0)
        st = lib().pt_get_vertices(self.handle, None, None, None, 0, ctypes.byref(n), 0)
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        V = int(n.value)
        S = ctypes.c_int64(0)
        st = lib().pt_get_tracks(self.handle, None, 0, ctypes.byref(S), 0)
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        out = np.zeros(V, VERTEX_DTYPE)
        off = np.empty(self.n_events + 1, np.int64)
        tv = np.empty(int(S.value), np.int32)
        _check(lib().pt_get_vertices(self.handle, _hptr(out), _hptr(off), _hptr(tv), V,
                                     ctypes.byref(n), 0))
        return out, off, tv

    def pt_get_cells(self):
        n = ctypes.c_int64(0)
        st = lib().pt_get_cells(self.handle, None, None, None, 0, ctypes.byref(n))
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        C = int(n.value)
        a, b, e = (np.empty(C, np.int32) for _ in range(3))
        _check(lib().pt_get_cells(self.handle, _hptr(a), _hptr(b), _hptr(e), C, ctypes.byref(n)))
        return a, b, e

    def pt_get_links(self):
        n = ctypes.c_int64(0)
        st = lib().pt_get_links(self.handle, None, None, None, None, None, 0, ctypes.byref(n))
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        Lk = int(n.value)
        h0, h1, h2, e = (np.empty(Lk, np.int32) for _ in range(4))
        q = np.empty(Lk, np.float32)
        _check(lib().pt_get_links(self.handle, _hptr(h0), _hptr(h1), _hptr(h2), _hptr(q),
                                  _hptr(e), Lk, ctypes.byref(n)))
        return h0, h1, h2, q, e

    def pt_get_candidates(self):
        n = ctypes.c_int64(0)
        st = lib().pt_get_candidates(self.handle, None, None, None, None, 0, ctypes.byref(n))
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        T = int(n.value)
        hits = np.empty((T, 6), np.int32)
        nh = np.empty(T, np.uint8)
        q = np.empty(T, np.float32)
        e = np.empty(T, np.int32)
        _check(lib().pt_get_candidates(self.handle, _hptr(hits), _hptr(nh), _hptr(q), _hptr(e),
                                       T, ctypes.byref(n)))
        return hits, nh, q, e

    def pt_set_launch(self, blocks_per_sm: int = 4, search_blocks_per_sm: int = 5):
        _check(lib().pt_set_launch(self.handle, int(blocks_per_sm), int(search_blocks_per_sm)))

    def pt_set_layer_pairs(self, pairs=None):
        """Layer pairs [(inner, outer), ...] for the doublets; None restores the default 13."""
        if not pairs:
            _check(lib().pt_set_layer_pairs(self.handle, 0, None, None))
            return
        a = np.ascontiguousarray([p[0] for p in pairs], np.int32)
        b = np.ascontiguousarray([p[1] for p in pairs], np.int32)
        _check(lib().pt_set_layer_pairs(self.handle, int(a.size), _hptr(a), _hptr(b)))

    def pt_set_wait_limit(self, cycles: int = 1 << 31):
        """Limit (SM cycles) of the context's bounded device-side waits."""
        _check(lib().pt_set_wait_limit(self.handle, int(cycles)))

    def pt_set_fishbone(self, on: bool = True):
        """Fishbone removal of aligned cells sharing an outer hit (off by default)."""
        _check(lib().pt_set_fishbone(self.handle, 1 if on else 0))

    def pt_debug_inject(self, site: int):
        """Debug build only: record a failure of bounds check `site` (reporting test)."""
        _check(lib().pt_debug_inject(self.handle, int(site)))

    def pt_set_tracing(self, on: bool = True):
        _check(lib().pt_set_tracing(self.handle, 1 if on else 0))

    def pt_get_trace(self) -> dict:
        """{kernel: (total ms, launches)} since the last call (tracing must be on)."""
        out = (PtKernelTime * 64)()
        n = ctypes.c_int(0)
        _check(lib().pt_get_trace(self.handle, out, 64, ctypes.byref(n)))
        return {out[i].name.decode(): (out[i].total_ms, int(out[i].launches))
                for i in range(n.value)}

    # -------------------------------------------------------------- learned gate
    def pt_set_gate(self, w, tau: float):
        """Enable the gate with 5057 float32 parameters (host), or disable it (w=None)."""
        if w is None:
            _check(lib().pt_set_gate(self.handle, None, 0.0))
            self.gate = None
            return
        arr = np.ascontiguousarray(w, np.float32)
        assert arr.size == 5057
        _check(lib().pt_set_gate(self.handle, _hptr(arr), float(tau)))
        self.gate = (arr.copy(), float(tau))

    def pt_get_link_features(self):
        """(feat float32 [n,12], h0, h1, h2, event int32 [n], score float32 [n])."""
        n = ctypes.c_int64(0)
        st = lib().pt_get_link_features(self.handle, None, None, None, None, None, None, 0,
                                        ctypes.byref(n))
        if st not in (PT_OK, PT_ERR_CAPACITY):
            _check(st)
        L = int(n.value)
        feat = np.empty((L, 12), np.float32)
        h0, h1, h2, e = (np.empty(L, np.int32) for _ in range(4))
        sc = np.empty(L, np.float32)
        _check(lib().pt_get_link_features(self.handle, _hptr(feat), _hptr(h0), _hptr(h1),
                                          _hptr(h2), _hptr(e), _hptr(sc), L, ctypes.byref(n)))
        return feat, h0, h1, h2, e, sc

    def pt_gate_score(self, feat_dev, out_dev):
        """Scores of device feature rows (torch float32 [n,12]) into out_dev [n]."""
        n = int(feat_dev.shape[0])
        _check(lib().pt_gate_score(self.handle, ctypes.c_void_p(feat_dev.data_ptr()), n,
                                   ctypes.c_void_p(out_dev.data_ptr())))

    # ------------------------------------------------------------ whole batch
    def pt_enqueue_batch(self, offsets, x, y, z, layer):
        off = np.ascontiguousarray(offsets, np.int64)
        px, dev, kx = _as_input(x, np.float32)
        py, _, ky = _as_input(y, np.float32)
        pz, _, kz = _as_input(z, np.float32)
        pl, _, kl = _as_input(layer, np.uint8)
        _check(lib().pt_enqueue_batch(self.handle, off.size - 1, _hptr(off), px, py, pz, pl, dev))
        self.n_events = off.size - 1

    def pt_reconstruct_batch(self, offsets, x, y, z, layer, out: dict | None = None):
        """Whole chain for a batch.  Returns (hits [S,6], nhits [S], tracks [S], offsets [E+1]).

        `out` may hold preallocated host arrays 'hits', 'nhits', 'tracks' (pinned ones are
        faster) of equal capacity, or torch CUDA tensors (then results stay on the device
        and the returned arrays are those tensors)."""
        off = np.ascontiguousarray(offsets, np.int64)
        E = off.size - 1
        px, dev, kx = _as_input(x, np.float32)
        py, _, ky = _as_input(y, np.float32)
        pz, _, kz = _as_input(z, np.float32)
        pl, _, kl = _as_input(layer, np.uint8)
        if out is None:
            capn = int(self.capacity["max_ntuplets"])
            out = dict(hits=np.empty((capn, 6), np.int32), nhits=np.empty(capn, np.uint8),
                       tracks=np.zeros(capn, TRACK_DTYPE))
        out_dev = int(hasattr(out["hits"], "is_cuda") and out["hits"].is_cuda)
        evoff = out.get("event_offsets")
        if evoff is None or evoff.shape[0] < E + 1:
            evoff = np.empty(E + 1, np.int64)
        n = ctypes.c_int64(0)
        _check(lib().pt_reconstruct_batch(
            self.handle, E, _hptr(off), px, py, pz, pl, dev,
            ctypes.c_void_p(_ptr_of(out["hits"])), ctypes.c_void_p(_ptr_of(out["nhits"])),
            ctypes.c_void_p(_ptr_of(out["tracks"])), ctypes.c_void_p(_ptr_of(evoff)),
            int(out["nhits"].shape[0]), ctypes.byref(n), out_dev))
        S = int(n.value)
        self.n_events = E
        return out["hits"][:S], out["nhits"][:S], out["tracks"][:S], evoff[: E + 1]


def _ptr_of(a) -> int:
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def exported_symbols() -> list[str]:
    """Names of EXPORTED found in the library (loads it; no GPU call)."""
    L = lib()
    return [s for s in EXPORTED if hasattr(L, s)]


def pt_gate_loss_grad(w, x, y, grad, loss, stream=None):
    """Mean BCE loss and gradient of the gate MLP; torch CUDA tensors (float32)."""
    sp = stream.cuda_stream if stream is not None else 0
    _check(lib().pt_gate_loss_grad(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), int(x.shape[0]),
                                   ctypes.c_void_p(grad.data_ptr()),
                                   ctypes.c_void_p(loss.data_ptr()),
                                   ctypes.c_void_p(sp) if sp else None))


def pt_gate_adam(w, m, v, grad, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on torch CUDA float32 tensors (in place)."""
    sp = stream.cuda_stream if stream is not None else 0
    _check(lib().pt_gate_adam(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                              ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                              int(w.numel()), float(lr), float(beta1), float(beta2), float(eps),
                              int(step), ctypes.c_void_p(sp) if sp else None))


class Server:
    """pt_server: continuous-batching request server (thread-safe)."""

    _fn = dict(submit="pt_submit", poll="pt_poll")

    def __init__(self, cuts: dict | None = None, budget_bytes: int = 2 << 30, slots: int = 2,
                 bfield: float = 3.8, device: int = 0):
        self.cuts = dict(cuts or default_cuts())
        h = ctypes.c_void_p(None)
        _check(lib().pt_server_create(
            ctypes.byref(PtGeometry(bfield)),
            ctypes.byref(PtCuts(*(float(self.cuts[k]) for k, _ in PtCuts._fields_))), device,
            int(budget_bytes), int(slots), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().pt_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def pt_server_set_gate(self, w, tau: float):
        arr = None if w is None else np.ascontiguousarray(w, np.float32)
        _check(lib().pt_server_set_gate(self.handle, None if arr is None else _hptr(arr),
                                        float(tau)))

    def pt_submit(self, x, y, z, layer) -> int:
        xs = [np.ascontiguousarray(a, t) for a, t in ((x, np.float32), (y, np.float32),
                                                     (z, np.float32), (layer, np.uint8))]
        t = ctypes.c_uint64(0)
        submit = getattr(lib(), self._fn["submit"])
        _check(submit(self.handle, xs[0].shape[0], *(_hptr(a) for a in xs), ctypes.byref(t)))
        return int(t.value)

    def pt_poll(self, ticket: int, timeout_us: int = -1):
        """(hits [S,6], nhits [S], tracks [S]); raises PtError (e.g. PT_ERR_NOT_READY)."""
        n = ctypes.c_int64(0)
        poll = getattr(lib(), self._fn["poll"])
        st = poll(self.handle, ticket, int(timeout_us), None, None, None, 0, ctypes.byref(n))
        if st == PT_OK:  # empty result, ticket released
            return (np.empty((0, 6), np.int32), np.empty(0, np.uint8), np.zeros(0, TRACK_DTYPE))
        if st != PT_ERR_CAPACITY:
            _check(st)
        S = int(n.value)
        hits = np.empty((S, 6), np.int32)
        nh = np.empty(S, np.uint8)
        tr = np.zeros(S, TRACK_DTYPE)
        _check(poll(self.handle, ticket, 0, _hptr(hits), _hptr(nh), _hptr(tr), S, ctypes.byref(n)))
        return hits, nh, tr

    def pt_server_stats(self) -> dict:
        p50, p99, eps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64(0)
        _check(lib().pt_server_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99),
                                     ctypes.byref(eps), ctypes.byref(n)))
        return dict(p50_ms=p50.value, p99_ms=p99.value, events_per_s=eps.value, n_done=n.value)

    def pt_server_counters(self) -> dict:
        b, s_, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pt_server_counters(self.handle, ctypes.byref(b), ctypes.byref(s_),
                                        ctypes.byref(r)))
        return dict(batches=b.value, split_batches=s_.value, requeued_events=r.value)

    def pt_server_reset_stats(self):
        _check(lib().pt_server_reset_stats(self.handle))


class Router(Server):
    """pt_router: several server instances behind one submit/poll front end."""

    _fn = dict(submit="pt_router_submit", poll="pt_router_poll")

    def __init__(self, instances: int = 2, cuts: dict | None = None,
                 budget_bytes_per_instance: int = 1 << 30, slots: int = 2, bfield: float = 3.8,
                 devices=None):
        self.cuts = dict(cuts or default_cuts())
        self.instances = int(instances)
        devs = np.ascontiguousarray(devices if devices is not None else [0] * self.instances,
                                    np.int32)
        h = ctypes.c_void_p(None)
        _check(lib().pt_router_create(
            ctypes.byref(PtGeometry(bfield)),
            ctypes.byref(PtCuts(*(float(self.cuts[k]) for k, _ in PtCuts._fields_))),
            _hptr(devs), self.instances, int(budget_bytes_per_instance), int(slots),
            ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().pt_router_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def pt_server_set_gate(self, w, tau: float):
        arr = None if w is None else np.ascontiguousarray(w, np.float32)
        _check(lib().pt_router_set_gate(self.handle, None if arr is None else _hptr(arr),
                                        float(tau)))

    def pt_server_stats(self) -> dict:
        p50, p99, eps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64(0)
        per = np.zeros(self.instances, np.int64)
        _check(lib().pt_router_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99),
                                     ctypes.byref(eps), ctypes.byref(n), _hptr(per)))
        return dict(p50_ms=p50.value, p99_ms=p99.value, events_per_s=eps.value, n_done=n.value,
                    per_instance=per.tolist())

    def pt_server_reset_stats(self):
        _check(lib().pt_router_reset_stats(self.handle))


def pt_autotune(offsets, x, y, z, layer, capacity: dict, phi_bins=(256, 512, 1024, 2048),
                blocks_per_sm=(2, 4, 8), search_blocks_per_sm=(3, 5, 8), reps: int = 3,
                cuts: dict | None = None, bfield: float = 3.8, device: int = 0) -> dict:
    """Fastest (phi_bins, blocks_per_sm, search_blocks_per_sm) for a sample batch given
    as host arrays; `table` maps "PxBxS" to the median chain time in ms (pt_ca.h)."""
    cuts = dict(cuts or default_cuts())
    off = np.ascontiguousarray(offsets, np.int64)
    arrs = [np.ascontiguousarray(a, t) for a, t in ((x, np.float32), (y, np.float32),
                                                    (z, np.float32), (layer, np.uint8))]
    pb, bp, sp = (np.ascontiguousarray(v, np.int32)
                  for v in (phi_bins, blocks_per_sm, search_blocks_per_sm))
    res = np.zeros(pb.size * bp.size * sp.size, np.float32)
    best = np.zeros(3, np.int32)
    _check(lib().pt_autotune(ctypes.byref(PtGeometry(bfield)),
                             ctypes.byref(PtCuts(*(float(cuts[k]) for k, _ in PtCuts._fields_))),
                             ctypes.byref(_cap(capacity)), device, off.size - 1, _hptr(off),
                             *(_hptr(a) for a in arrs), _hptr(pb), pb.size, _hptr(bp), bp.size,
                             _hptr(sp), sp.size, int(reps), _hptr(best), _hptr(res)))
    keys = [f"{int(p)}x{int(b)}x{int(q)}" for p in pb for b in bp for q in sp]
    return dict(phi_bins=int(best[0]), blocks_per_sm=int(best[1]),
                search_blocks_per_sm=int(best[2]),
                table={k: round(float(v), 4) for k, v in zip(keys, res)})
