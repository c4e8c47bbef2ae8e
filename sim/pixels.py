"""Synthetic pixel readout of the generated hits (input recipe only).

Every detector surface is divided into modules (barrel: sectors in phi x segments in
z; disks: sectors in phi x rings in r) with a rectangular pixel grid in (phi, z) or
(phi, r), read from params/pixels_v1.json.  A hit deposits a fixed charge spread
uniformly over a square cloud one pixel wide centred on it; each pixel collects the
charge of the part of the cloud it covers, charges of the same pixel add up, and a
pixel whose charge rounded down reaches the threshold is read out as a digi
(module, row, col, adc).  The raw event is the list of digis grouped by module, in the
order the modules are first hit, packed one digi per 64-bit word:
module << 40 | row << 28 | col << 16 | adc.  No reconstruction arithmetic lives here:
turning digis back into hits is the library's job (and the oracle's).
"""

from __future__ import annotations

import json
import math
import os

import numpy as np

from .events import Event

_PARAMS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2501_05520_gb300", "params", "pixels_v1.json")


def load_params(path: str = _PARAMS) -> dict:
    with open(path) as f:
        return json.load(f)


def module_table(params: dict | None = None) -> dict:
    """Modules in index order (barrel layers 0-3, then disks 4-9; sector-major), as
    float64 arrays: layer, kind (0 barrel, 1 disk), rz (barrel radius or disk z),
    phi0, dphi_col (angle per column), v0, dv_row (cm per row), ncol, nrow."""
    p = params or load_params()
    rows = []
    b = p["barrel"]
    dz = (b["zmax"] - b["zmin"]) / b["segments"]
    for L, (r, S) in enumerate(zip(b["r"], b["sectors"])):
        dphi = 2.0 * math.pi / S
        ncol = math.ceil(r * dphi / p["pitch_rphi"])
        nrow = math.ceil(dz / p["pitch_z"])
        for s in range(S):
            for g in range(b["segments"]):
                rows.append((L, 0, r, -math.pi + s * dphi, dphi / ncol, b["zmin"] + g * dz,
                             p["pitch_z"], ncol, nrow))
    d = p["disks"]
    dr = (d["rmax"] - d["rmin"]) / d["rings"]
    for side, base in ((1.0, 4), (-1.0, 7)):
        for k, zd in enumerate(d["z"]):
            dphi = 2.0 * math.pi / d["sectors"]
            for s in range(d["sectors"]):
                for g in range(d["rings"]):
                    rmid = d["rmin"] + (g + 0.5) * dr
                    ncol = math.ceil(rmid * dphi / p["pitch_rphi"])
                    rows.append((base + k, 1, side * zd, -math.pi + s * dphi, dphi / ncol,
                                 d["rmin"] + g * dr, p["pitch_r"], ncol,
                                 math.ceil(dr / p["pitch_r"])))
    a = np.asarray(rows, np.float64)
    names = ("layer", "kind", "rz", "phi0", "dphi_col", "v0", "dv_row", "ncol", "nrow")
    return {n: a[:, i] for i, n in enumerate(names)}


def _module_of(mt: dict, p: dict, layer: np.ndarray, phi: np.ndarray, v: np.ndarray):
    """Module index of points on their layer's surface."""
    b, d = p["barrel"], p["disks"]
    first = np.zeros(10, np.int64)
    nmod = np.zeros(10, np.int64)
    off = 0
    for L, S in enumerate(b["sectors"]):
        first[L], nmod[L] = off, S * b["segments"]
        off += S * b["segments"]
    for L in range(4, 10):
        first[L], nmod[L] = off, d["sectors"] * d["rings"]
        off += d["sectors"] * d["rings"]
    barrel = layer < 4
    S = np.where(barrel, np.asarray(b["sectors"] + [d["sectors"]] * 6)[layer], d["sectors"])
    G = np.where(barrel, b["segments"], d["rings"])
    s = np.clip(np.floor((phi + math.pi) / (2.0 * math.pi) * S).astype(np.int64), 0, S - 1)
    lo = np.where(barrel, b["zmin"], d["rmin"])
    hi = np.where(barrel, b["zmax"], d["rmax"])
    g = np.clip(np.floor((v - lo) / (hi - lo) * G).astype(np.int64), 0, G - 1)
    return first[layer] + s * G + g


def digitize(ev: Event, params: dict | None = None):
    """Raw digis of one event: (uint64 words, int64 [n] source hit of each digi's
    largest charge, module table).  Uses the float64 hit positions."""
    p = params or load_params()
    mt = module_table(p)
    q = p["charge"]
    layer = ev.layer.astype(np.int64)
    x, y, z = ev.x64, ev.y64, ev.z64
    phi = np.arctan2(y, x)
    r = np.hypot(x, y)
    v = np.where(layer < 4, z, r)
    mod = _module_of(mt, p, layer, phi, v)
    dphi = phi - mt["phi0"][mod]
    dphi = np.where(dphi < 0, dphi + 2.0 * math.pi, dphi)
    a = dphi / mt["dphi_col"][mod]            # cloud centre in pixel units
    bv = (v - mt["v0"][mod]) / mt["dv_row"][mod]
    w = q["cloud_pixels"]
    charge = {}
    src = {}
    for h in range(layer.size):
        m = int(mod[h])
        ncol, nrow = int(mt["ncol"][m]), int(mt["nrow"][m])
        a0, a1 = a[h] - 0.5 * w, a[h] + 0.5 * w
        b0, b1 = bv[h] - 0.5 * w, bv[h] + 0.5 * w
        for col in range(max(0, math.floor(a0)), min(ncol - 1, math.floor(a1)) + 1):
            ou = (min(a1, col + 1.0) - max(a0, float(col))) / w
            if ou <= 0:
                continue
            for row in range(max(0, math.floor(b0)), min(nrow - 1, math.floor(b1)) + 1):
                ov = (min(b1, row + 1.0) - max(b0, float(row))) / w
                if ov <= 0:
                    continue
                key = (m, row, col)
                c = q["adc_per_hit"] * ou * ov
                charge[key] = charge.get(key, 0.0) + c
                if c > src.get(key, (-1.0, -1))[0]:
                    src[key] = (c, h)
    # group by module in the order modules are first hit, pixels in (row, col) order
    first_hit = {}
    for h in range(layer.size):
        first_hit.setdefault(int(mod[h]), h)
    words, owner = [], []
    by_mod = {}
    for (m, row, col), c in charge.items():
        adc = int(math.floor(c))
        if adc >= q["threshold_adc"]:
            by_mod.setdefault(m, []).append((row, col, min(adc, 65535), src[(m, row, col)][1]))
    for m in sorted(by_mod, key=lambda k: first_hit[k]):
        for row, col, adc, h in sorted(by_mod[m]):
            words.append((m << 40) | (row << 28) | (col << 16) | adc)
            owner.append(h)
    return np.asarray(words, np.uint64), np.asarray(owner, np.int64), mt


def unpack(words: np.ndarray):
    """(module, row, col, adc) int64 arrays of packed digis."""
    w = np.asarray(words, np.uint64)
    return ((w >> np.uint64(40)).astype(np.int64), ((w >> np.uint64(28)) & np.uint64(0xfff)).astype(np.int64),
            ((w >> np.uint64(16)) & np.uint64(0xfff)).astype(np.int64), (w & np.uint64(0xffff)).astype(np.int64))


def concat_raw(raws):
    """Batch layout of several events' digis: (offsets int64 [E+1], words uint64)."""
    off = np.zeros(len(raws) + 1, np.int64)
    off[1:] = np.cumsum([w.size for w in raws])
    return off, (np.concatenate(raws) if raws else np.zeros(0, np.uint64))
