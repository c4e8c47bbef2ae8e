"""CPU oracle for raw pixel data -> hits (digi unpacking, clustering, hit positions).

TEST INFRASTRUCTURE ONLY: the tests are the only callers; the product never loads it.
It shares no code with the CUDA path (it builds its own module table from the same
parameter file, read as data).

The paper's chain starts from compressed raw data that the GPU unpacks into "digis";
neighbouring digis of one detector layer are clustered and each cluster gives a hit
(Sec. 2.2.1 and the caption of Fig. 2).  It fixes no format or algorithm; this
library's reading:

  [P1] A digi is (module, row, col, adc), packed in 64 bits as
       module << 40 | row << 28 | col << 16 | adc; an event's digis come grouped by
       module, and a pixel appears at most once.
  [P2] A cluster is a set of digis of one module connected through pixels that touch
       at an edge or a corner (8-neighbourhood).
  [P3] Its hit lies at the adc-weighted mean pixel centre: col_c = sum adc (col + 1/2)
       / sum adc, row_c likewise; phi = phi0 + col_c dphi_col and v = v0 + row_c
       dv_row; a barrel module gives (r cos phi, r sin phi, v), a disk module
       (v cos phi, v sin phi, z).  The hit's layer is the module's.
  [P4] Hits of an event come module run by module run in input order, and within a
       module in order of their cluster's first pixel in (row, col) order.

Arithmetic is float64; the adc sums are exact integers.
"""

from __future__ import annotations

import json
import math

import numpy as np

MODULE_FIELDS = ("layer", "kind", "rz", "phi0", "dphi_col", "v0", "dv_row", "ncol", "nrow")


def modules(path: str) -> np.ndarray:
    """Module table [M, 9] (MODULE_FIELDS) in module-index order: barrel layers 0..3,
    then the +z disks (layers 4..6) and the -z disks (7..9); within a layer, sector by
    sector (phi from -pi), and within a sector segment by segment (z) or ring by ring
    (r).  Barrel: sectors of 2 pi / S, segments of (zmax - zmin) / G, ncol = ceil(r x
    sector angle / pitch_rphi), nrow = ceil(segment length / pitch_z).  Disks: rings of
    (rmax - rmin) / R, ncol = ceil(ring-centre radius x sector angle / pitch_rphi),
    nrow = ceil(ring width / pitch_r).  The column angle is the sector angle / ncol."""
    with open(path) as f:
        p = json.load(f)
    out = []
    b = p["barrel"]
    seg = (b["zmax"] - b["zmin"]) / b["segments"]
    for L in range(len(b["r"])):
        r, S = b["r"][L], b["sectors"][L]
        ang = 2.0 * math.pi / S
        ncol, nrow = math.ceil(r * ang / p["pitch_rphi"]), math.ceil(seg / p["pitch_z"])
        for s in range(S):
            for g in range(b["segments"]):
                out.append([L, 0, r, -math.pi + s * ang, ang / ncol, b["zmin"] + g * seg,
                            p["pitch_z"], ncol, nrow])
    d = p["disks"]
    ring = (d["rmax"] - d["rmin"]) / d["rings"]
    ang = 2.0 * math.pi / d["sectors"]
    for L in range(4, 10):
        zd = d["z"][(L - 4) % 3] * (1.0 if L < 7 else -1.0)
        for s in range(d["sectors"]):
            for g in range(d["rings"]):
                ncol = math.ceil((d["rmin"] + (g + 0.5) * ring) * ang / p["pitch_rphi"])
                out.append([L, 1, zd, -math.pi + s * ang, ang / ncol, d["rmin"] + g * ring,
                            p["pitch_r"], ncol, math.ceil(ring / p["pitch_r"])])
    return np.asarray(out, np.float64)


def decode(words) -> tuple:
    """[P1] (module, row, col, adc) of packed digis."""
    w = [int(v) for v in np.asarray(words, np.uint64)]
    return (np.asarray([v >> 40 for v in w], np.int64),
            np.asarray([(v >> 28) & 0xfff for v in w], np.int64),
            np.asarray([(v >> 16) & 0xfff for v in w], np.int64),
            np.asarray([v & 0xffff for v in w], np.int64))


def _components(rows, cols):
    """[P2] 8-connected components of one module's pixels; labels = smallest member
    index in (row, col) order."""
    n = len(rows)
    parent = list(range(n))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    at = {(int(r), int(c)): i for i, (r, c) in enumerate(zip(rows, cols))}
    for i in range(n):
        r, c = int(rows[i]), int(cols[i])
        for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
            j = at.get((r + dr, c + dc))
            if j is not None:
                a, b = find(i), find(j)
                if a != b:
                    parent[max(a, b)] = min(a, b)
    return [find(i) for i in range(n)]


def reconstruct(words, table: np.ndarray):
    """Hits of one event's raw digis: (x, y, z float64 [H], layer int64 [H],
    members: list of H arrays of digi indices)."""
    mod, row, col, adc = decode(words)
    n = mod.size
    # [P1] module runs in input order
    starts = [0] + [i for i in range(1, n) if mod[i] != mod[i - 1]] + [n]
    xs, ys, zs, ls, members = [], [], [], [], []
    for a, b in zip(starts[:-1], starts[1:]):
        if b <= a:
            continue
        idx = np.arange(a, b)
        order = idx[np.lexsort((col[idx], row[idx]))]  # (row, col) order
        lab = _components(row[order], col[order])
        m = table[int(mod[a])]
        groups = {}
        for k, root in enumerate(lab):
            groups.setdefault(root, []).append(order[k])
        for root in sorted(groups):  # [P4] by the cluster's first pixel
            g = np.asarray(groups[root], np.int64)
            wsum = int(adc[g].sum())
            col_c = float(np.sum(adc[g] * (2 * col[g] + 1))) / (2.0 * wsum)
            row_c = float(np.sum(adc[g] * (2 * row[g] + 1))) / (2.0 * wsum)
            phi = m[3] + col_c * m[4]
            v = m[5] + row_c * m[6]
            if m[1] == 0:  # [P3] barrel
                xs.append(m[2] * math.cos(phi)); ys.append(m[2] * math.sin(phi)); zs.append(v)
            else:
                xs.append(v * math.cos(phi)); ys.append(v * math.sin(phi)); zs.append(m[2])
            ls.append(int(m[0]))
            members.append(np.sort(g))
    return (np.asarray(xs), np.asarray(ys), np.asarray(zs), np.asarray(ls, np.int64), members)


def components_brute_force(rows, cols):
    """Pixel groups by breadth-first search over all pairs (|dr| <= 1 and |dc| <= 1):
    the definition of [P2] on small inputs, to pin _components."""
    n = len(rows)
    seen = [False] * n
    groups = []
    for s in range(n):
        if seen[s]:
            continue
        seen[s] = True
        stack, g = [s], []
        while stack:
            i = stack.pop()
            g.append(i)
            for j in range(n):
                if not seen[j] and abs(int(rows[i]) - int(rows[j])) <= 1 and \
                        abs(int(cols[i]) - int(cols[j])) <= 1:
                    seen[j] = True
                    stack.append(j)
        groups.append(sorted(g))
    return sorted(groups)
