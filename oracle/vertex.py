"""CPU oracle for primary-vertex reconstruction from fitted tracks.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU-baseline leg are the only
callers; the product never loads it.  It shares no code with the CUDA path.

The paper lists vertex reconstruction as the last of Patatrack's sub-algorithms and
has the chain hand back vertices along with the tracks (Sec. 2.2.1 and the caption
of Fig. 2); it gives no algorithm.  This library's reading (the
plain definition the GPU must reproduce):

  [V1] The input of an event is its cleaned, fitted tracks with at least `min_hits`
       hits (default 4: quadruplets and longer, whose z0 is measured by at least two
       cells) and a finite z0.
  [V2] The tracks are put in order of z0 (ties: the track's position in the event's
       canonical order), and the ordered list is cut wherever the step from one z0 to
       the next exceeds `dz` (a step of exactly dz does not cut).  This is
       single-linkage clustering in z0 at distance dz.
  [V3] Every group of at least two tracks is a vertex: z = mean z0 of its tracks,
       sum_pt2 = sum of their pT squared, n = their number.  Vertices come in order of
       z, and every used track records its vertex.

Arithmetic is float64 throughout; `find_vertices` follows the three steps in order.
"""

from __future__ import annotations

import numpy as np

DZ_DEFAULT = 0.02  # cm: above the z0 resolution of a quadruplet, below the vertex spacing
MIN_HITS_DEFAULT = 4


def find_vertices(z0, pt, nhits, min_hits: int = MIN_HITS_DEFAULT, dz: float = DZ_DEFAULT):
    """Vertices of one event's tracks ([V1]-[V3]).

    z0, pt, nhits: per-track arrays in the event's canonical track order.
    Returns (vertices, track_vertex): vertices is a float64 array [V, 3] of
    (z, sum_pt2, n) in order of z; track_vertex is int64 [T], the vertex of each track
    or -1.
    """
    z0 = np.asarray(z0, np.float64)
    pt = np.asarray(pt, np.float64)
    nhits = np.asarray(nhits)
    T = z0.shape[0]
    track_vertex = np.full(T, -1, np.int64)
    # [V1] the tracks that take part
    used = np.nonzero((nhits >= min_hits) & np.isfinite(z0))[0]
    if used.size == 0:
        return np.zeros((0, 3)), track_vertex
    # [V2] order by z0, ties by position; cut where the step exceeds dz
    order = used[np.lexsort((used, z0[used]))]
    zs = z0[order]
    starts = np.concatenate([[0], np.nonzero(np.diff(zs) > dz)[0] + 1, [zs.size]])
    # [V3] groups of at least two tracks
    vertices = []
    for a, b in zip(starts[:-1], starts[1:]):
        if b - a < 2:
            continue
        members = order[a:b]
        track_vertex[members] = len(vertices)
        vertices.append((zs[a:b].mean(), float(np.sum(pt[members] ** 2)), float(b - a)))
    return np.asarray(vertices, np.float64).reshape(-1, 3), track_vertex


def single_linkage_groups(z0, dz: float):
    """Brute-force single-linkage groups of a small list of values: two values are in
    one group iff a chain of values links them, each step at most dz.  O(n^2) union
    find, used to pin find_vertices' sort-and-cut against the definition."""
    z0 = np.asarray(z0, np.float64)
    n = z0.shape[0]
    parent = list(range(n))

    def root(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for i in range(n):
        for j in range(i + 1, n):
            if abs(z0[i] - z0[j]) <= dz:
                parent[root(i)] = root(j)
    groups = {}
    for i in range(n):
        groups.setdefault(root(i), []).append(i)
    return sorted((sorted(g) for g in groups.values()), key=lambda g: min(z0[g]))
