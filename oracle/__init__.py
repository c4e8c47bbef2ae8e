"""CPU oracle for the pixel-track cellular automaton.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg are the only callers.  The product (the CUDA library and its binding) never loads
it.  It shares no code with the CUDA path; see oracle.c for what each stage computes.

Wrapper layout: `build()` compiles oracle.c with gcc (-O2 -ffp-contract=off, no fast
math) into liboracle.so next to this file; `reconstruct()` runs the whole chain on one
event and returns numpy arrays; `fit_hits()` fits one hit list.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FIT_FIELDS = ("kappa", "phi0", "d0", "cot_theta", "z0", "pt", "chi2_circle", "chi2_line",
              "charge")

# The chain's (inner, outer) layer pairs: consecutive surfaces a primary track can cross.
DEFAULT_PAIRS = ((0, 1), (1, 2), (2, 3), (0, 4), (1, 4), (2, 4), (4, 5), (5, 6),
                 (0, 7), (1, 7), (2, 7), (7, 8), (8, 9))


def gap_pairs(pairs=DEFAULT_PAIRS) -> tuple:
    """[L1] Skip-layer pairs: (a, c) for every two-step path a -> b -> c of the pair graph
    that is not itself a pair (a track that misses the surface b still joins a and c),
    in (a, c) order."""
    allowed = set(pairs)
    out = {(a, c) for a, b in pairs for b2, c in pairs if b2 == b and (a, c) not in allowed}
    return tuple(sorted(out))


class Cuts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_float), ("z0max", ctypes.c_float), ("cotmax", ctypes.c_float),
                ("rz0", ctypes.c_float), ("rz1", ctypes.c_float), ("dca_b0", ctypes.c_float),
                ("dca_other", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, float32 without FMA contraction, float64 fit)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cc = os.environ.get("CC", "gcc")
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.orc_reconstruct.restype = P
        lib.orc_reconstruct.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.POINTER(Cuts),
                                        ctypes.c_double]
        lib.orc_reconstruct_masked.restype = P
        lib.orc_reconstruct_masked.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.POINTER(Cuts),
                                               ctypes.c_double, P, ctypes.c_int64]
        lib.orc_reconstruct_pairs.restype = P
        lib.orc_reconstruct_pairs.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.POINTER(Cuts),
                                              ctypes.c_double, ctypes.c_int, P, P]
        lib.orc_reconstruct_ex.restype = P
        lib.orc_reconstruct_ex.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.POINTER(Cuts),
                                           ctypes.c_double, ctypes.c_int, P, P, P,
                                           ctypes.c_int64, ctypes.c_int]
        for name in ("orc_sizes", "orc_get_radius", "orc_get_near"):
            getattr(lib, name).argtypes = [P, P]
        lib.orc_get_cells.argtypes = [P, P, P]
        lib.orc_get_links.argtypes = [P, P, P, P]
        lib.orc_get_ntuplets.argtypes = [P, P, P, P, P]
        lib.orc_get_survivors.argtypes = [P, P, P]
        lib.orc_free.argtypes = [P]
        lib.orc_fit_hits.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P]
        lib.orc_doublet_ok.argtypes = [ctypes.POINTER(Cuts), P, P, P]
        lib.orc_link_ok.argtypes = [ctypes.POINTER(Cuts), P, ctypes.c_int, P, P, P, P]
        lib.orc_fb_loses.argtypes = [P, P, ctypes.c_int, ctypes.c_int64, P, ctypes.c_int,
                                     ctypes.c_int64]
        lib.orc_dedup.restype = ctypes.c_int64
        lib.orc_dedup.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64, ctypes.c_int64, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_cuts(d: dict) -> Cuts:
    return Cuts(*(float(np.float32(d[f])) for f, _ in Cuts._fields_))


def reconstruct(x, y, z, layer, cuts: dict, bfield: float = 3.8, link_keep=None,
                pairs=None, fishbone: bool = False) -> dict:
    """Run the whole chain on one event.  Hit arrays are float32 / uint8, input order.

    link_keep: optional bool array, one entry per link of the plain run (its link order);
    links with False are removed before the ntuplet search (a gate decision).
    pairs: optional (inner, outer) layer-pair table replacing DEFAULT_PAIRS (e.g.
    DEFAULT_PAIRS + gap_pairs()).
    fishbone: apply the fishbone step (aligned active cells sharing an outer hit) to the
    links before the ntuplet search; the returned links are those that remain.

    Returns a dict of numpy arrays:
      r                      float32 [N]
      cell_inner, cell_outer int32 [C]      input hit indices
      link_a, link_b         int32 [L]      cell indices;  link_q float32 [L]
      nt_hits int32 [T,6] (-1 pad), nt_cells int32 [T,5], nt_n int32 [T], nt_q float32 [T]
      survivors int32 [S]    indices into nt_*, canonical order (hit tuple ascending)
      fit float64 [S,9]      FIT_FIELDS per survivor
      near int32 [K,4]       near-threshold decisions (kind, h0, h1, h2)
      n_doublet_tests, n_link_tests
    """
    lib = _load()
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    layer = np.ascontiguousarray(layer, np.uint8)
    n = x.shape[0]
    c = make_cuts(cuts)
    if pairs is not None:
        pt = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2).T)
        pin, pout = np.ascontiguousarray(pt[0]), np.ascontiguousarray(pt[1])
        if pin.size == 0:
            raise ValueError("invalid layer-pair table")
    else:
        pin = pout = np.zeros(0, np.int32)
    keep = None if link_keep is None else np.ascontiguousarray(link_keep, np.uint8)
    h = lib.orc_reconstruct_ex(n, _ptr(x), _ptr(y), _ptr(z), _ptr(layer), ctypes.byref(c),
                               float(bfield), int(pin.size), _ptr(pin), _ptr(pout),
                               _ptr(keep) if keep is not None else None,
                               0 if keep is None else keep.size, int(bool(fishbone)))
    if not h:
        raise ValueError("invalid layer-pair table")
    try:
        sz = np.zeros(7, np.int64)
        lib.orc_sizes(h, _ptr(sz))
        C, L, T, S, K = (int(v) for v in sz[:5])
        out = dict(r=np.empty(n, np.float32),
                   cell_inner=np.empty(C, np.int32), cell_outer=np.empty(C, np.int32),
                   link_a=np.empty(L, np.int32), link_b=np.empty(L, np.int32),
                   link_q=np.empty(L, np.float32),
                   nt_hits=np.empty((T, 6), np.int32), nt_cells=np.empty((T, 5), np.int32),
                   nt_n=np.empty(T, np.int32), nt_q=np.empty(T, np.float32),
                   survivors=np.empty(S, np.int32), fit=np.empty((S, 9), np.float64),
                   near=np.empty((K, 4), np.int32),
                   n_doublet_tests=int(sz[5]), n_link_tests=int(sz[6]))
        lib.orc_get_radius(h, _ptr(out["r"]))
        lib.orc_get_cells(h, _ptr(out["cell_inner"]), _ptr(out["cell_outer"]))
        lib.orc_get_links(h, _ptr(out["link_a"]), _ptr(out["link_b"]), _ptr(out["link_q"]))
        lib.orc_get_ntuplets(h, _ptr(out["nt_hits"]), _ptr(out["nt_cells"]), _ptr(out["nt_n"]),
                             _ptr(out["nt_q"]))
        lib.orc_get_survivors(h, _ptr(out["survivors"]), _ptr(out["fit"]))
        lib.orc_get_near(h, _ptr(out["near"]))
    finally:
        lib.orc_free(h)
    return out


def survivors_hits(res: dict) -> np.ndarray:
    """Surviving ntuplets as an int32 [S,6] array of input hit indices (-1 pad), canonical order."""
    return res["nt_hits"][res["survivors"]]


def fit_hits(x, y, z, bfield: float = 3.8) -> np.ndarray:
    """Float64 circle + line fit of one hit list (inner to outer).  Returns FIT_FIELDS."""
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.zeros(9, np.float64)
    lib.orc_fit_hits(int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), float(bfield), _ptr(out))
    return out


def doublet_ok(cuts: dict, hi, ho):
    """Single doublet decision (inner hit hi, outer hit ho as float32 (x, y, z))."""
    lib = _load()
    a = np.ascontiguousarray(hi, np.float32)
    b = np.ascontiguousarray(ho, np.float32)
    near = ctypes.c_int(0)
    c = make_cuts(cuts)
    ok = lib.orc_doublet_ok(ctypes.byref(c), _ptr(a), _ptr(b), ctypes.byref(near))
    return bool(ok), bool(near.value)


def link_ok(cuts: dict, h0, layer0: int, h1, h2):
    """Single link decision for hits h0 -> h1 -> h2 (float32 (x, y, z)); returns (ok, near, q)."""
    lib = _load()
    a = np.ascontiguousarray(h0, np.float32)
    b = np.ascontiguousarray(h1, np.float32)
    d = np.ascontiguousarray(h2, np.float32)
    near = ctypes.c_int(0)
    q = ctypes.c_float(0)
    c = make_cuts(cuts)
    ok = lib.orc_link_ok(ctypes.byref(c), _ptr(a), int(layer0), _ptr(b), _ptr(d),
                         ctypes.byref(near), ctypes.byref(q))
    return bool(ok), bool(near.value), float(q.value)


def fishbone_loses(h, i, layer_i: int, key_i: int, j, layer_j: int, key_j: int) -> bool:
    """The fishbone comparison: does cell (i -> h) lose to cell (j -> h)?  h, i, j are
    (x, y, z) points, rounded to float32."""
    lib = _load()
    a = [np.ascontiguousarray(v, np.float32) for v in (h, i, j)]
    return bool(lib.orc_fb_loses(_ptr(a[0]), _ptr(a[1]), int(layer_i), int(key_i), _ptr(a[2]),
                                 int(layer_j), int(key_j)))


def dedup(hits, cells, nh, q, n_cells: int, n_hits: int) -> np.ndarray:
    """Duplicate cleaning of a given ntuplet list; returns survivor indices, canonical order."""
    lib = _load()
    hits = np.ascontiguousarray(hits, np.int32).reshape(-1, 6)
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 5)
    nh = np.ascontiguousarray(nh, np.int32)
    q = np.ascontiguousarray(q, np.float32)
    T = nh.shape[0]
    out = np.zeros(max(T, 1), np.int32)
    S = lib.orc_dedup(T, _ptr(hits), _ptr(cells), _ptr(nh), _ptr(q), int(n_cells), int(n_hits),
                      _ptr(out))
    return out[:S].copy()
