"""Pixel-readout module table of the library's detector (params/pixels_v1.json).

Builds the pt_module array that pt_set_modules preloads: barrel layers 0..3 (at radius
r, sectors of 2 pi / S in phi x segments of the z range), then the +z disks (layers
4..6) and the -z disks (7..9) (sectors x rings of the r range); modules in that order,
sector by sector (phi from -pi), segment / ring within a sector.  Columns run along phi
(ceil(radius x sector angle / pitch_rphi) of them, the radius being the ring centre on
disks), rows along z or r (ceil(extent / pitch)).
"""

from __future__ import annotations

import json
import math
import os

import numpy as np

PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "params", "pixels_v1.json")

MODULE_DTYPE = np.dtype([("layer", "<i4"), ("kind", "<i4"), ("rz", "<f4"), ("phi0", "<f4"),
                         ("dphi_col", "<f4"), ("v0", "<f4"), ("dv_row", "<f4"), ("ncol", "<i4"),
                         ("nrow", "<i4")])
assert MODULE_DTYPE.itemsize == 36


def module_table(path: str = PARAMS) -> np.ndarray:
    with open(path) as f:
        p = json.load(f)
    mods = []
    b, d = p["barrel"], p["disks"]
    seg = (b["zmax"] - b["zmin"]) / b["segments"]
    for layer, (r, sectors) in enumerate(zip(b["r"], b["sectors"])):
        ang = 2.0 * math.pi / sectors
        ncol = math.ceil(r * ang / p["pitch_rphi"])
        for s in range(sectors):
            for g in range(b["segments"]):
                mods.append((layer, 0, r, -math.pi + s * ang, ang / ncol, b["zmin"] + g * seg,
                             p["pitch_z"], ncol, math.ceil(seg / p["pitch_z"])))
    ring = (d["rmax"] - d["rmin"]) / d["rings"]
    ang = 2.0 * math.pi / d["sectors"]
    for layer in range(4, 10):
        zd = d["z"][(layer - 4) % 3] * (1.0 if layer < 7 else -1.0)
        for s in range(d["sectors"]):
            for g in range(d["rings"]):
                ncol = math.ceil((d["rmin"] + (g + 0.5) * ring) * ang / p["pitch_rphi"])
                mods.append((layer, 1, zd, -math.pi + s * ang, ang / ncol, d["rmin"] + g * ring,
                             p["pitch_r"], ncol, math.ceil(ring / p["pitch_r"])))
    return np.asarray(mods, MODULE_DTYPE)
