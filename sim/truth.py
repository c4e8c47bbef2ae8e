"""Generator-truth bookkeeping for efficiency, fake and duplicate rates.

Definitions (the paper prints none; these are the library's evaluation readings):
  reconstructable particle: >= 3 hits forming a chain of consecutive surfaces on
      allowed layer pairs (the longest such chain along the track has >= 3 hits);
  matched ntuplet: all of its hits come from one particle (a >= 75 % variant too);
  efficiency: reconstructable particles matched by >= 1 ntuplet / reconstructable;
  fake rate: unmatched ntuplets / ntuplets;
  duplicate rate: reconstructable particles matched more than once / reconstructable.
"""

from __future__ import annotations

import numpy as np

# Allowed (inner, outer) layer pairs of the detector (layer codes as in sim.events).
LAYER_PAIRS = ((0, 1), (1, 2), (2, 3), (0, 4), (1, 4), (2, 4), (4, 5), (5, 6),
               (0, 7), (1, 7), (2, 7), (7, 8), (8, 9))
_ALLOWED = set(LAYER_PAIRS)
# order of the surfaces along an outgoing track
_DEPTH = np.array([0, 1, 2, 3, 4, 5, 6, 4, 5, 6])


def particle_chains(pid: np.ndarray, layer: np.ndarray, pairs=LAYER_PAIRS) -> dict:
    """Per particle: its hits ordered along the track, and the longest chain of hits whose
    consecutive layers are pairs of `pairs`."""
    allowed = _ALLOWED if pairs is LAYER_PAIRS else set(map(tuple, pairs))
    out = {}
    order = np.argsort(pid, kind="stable")
    ps = pid[order]
    bounds = np.flatnonzero(np.diff(ps)) + 1
    for grp in np.split(order, bounds):
        if grp.size == 0 or pid[grp[0]] < 0:
            continue
        hits = grp[np.argsort(_DEPTH[layer[grp]], kind="stable")]
        best, cur = [hits[0]], [hits[0]]
        for h in hits[1:]:
            if (int(layer[cur[-1]]), int(layer[h])) in allowed:
                cur.append(h)
            else:
                cur = [h]
            if len(cur) > len(best):
                best = list(cur)
        out[int(pid[grp[0]])] = dict(hits=hits, chain=np.asarray(best))
    return out


def match(ntuplets: np.ndarray, pid: np.ndarray, frac: float = 1.0) -> np.ndarray:
    """Matched particle per ntuplet (-1 if none).  ntuplets: int [T,6], -1 padded."""
    T = ntuplets.shape[0]
    res = np.full(T, -1, np.int64)
    for t in range(T):
        h = ntuplets[t][ntuplets[t] >= 0]
        p = pid[h]
        vals, cnt = np.unique(p[p >= 0], return_counts=True)
        if vals.size and cnt.max() >= frac * h.size - 1e-9:
            res[t] = vals[np.argmax(cnt)]
    return res


def rates(ntuplets: np.ndarray, pid: np.ndarray, layer: np.ndarray, frac: float = 1.0) -> dict:
    """Efficiency, fake rate and duplicate rate of an ntuplet set against truth."""
    chains = particle_chains(pid, layer)
    reco = {p for p, c in chains.items() if c["chain"].size >= 3}
    m = match(ntuplets, pid, frac)
    matched_p, counts = np.unique(m[m >= 0], return_counts=True)
    cnt = dict(zip(matched_p.tolist(), counts.tolist()))
    n_reco = len(reco)
    eff = sum(1 for p in reco if p in cnt) / max(n_reco, 1)
    dup = sum(1 for p in reco if cnt.get(p, 0) > 1) / max(n_reco, 1)
    fake = float(np.mean(m < 0)) if m.size else 0.0
    return dict(efficiency=eff, fake_rate=fake, duplicate_rate=dup, n_reconstructable=n_reco,
                n_ntuplets=int(ntuplets.shape[0]), n_fake=int(np.sum(m < 0)))


def true_doublets(pid: np.ndarray, layer: np.ndarray):
    """(inner, outer) hit pairs that are consecutive hits of one particle on an allowed pair."""
    pairs = []
    for c in particle_chains(pid, layer).values():
        h = c["hits"]
        for a, b in zip(h[:-1], h[1:]):
            if (int(layer[a]), int(layer[b])) in _ALLOWED:
                pairs.append((a, b))
    return np.asarray(pairs, np.int64).reshape(-1, 2)


def true_triplets(pid: np.ndarray, layer: np.ndarray):
    """Consecutive hit triples of one particle whose two doublets are on allowed pairs."""
    tri = []
    for c in particle_chains(pid, layer).values():
        h = c["hits"]
        for a, b, d in zip(h[:-2], h[1:-1], h[2:]):
            if ((int(layer[a]), int(layer[b])) in _ALLOWED
                    and (int(layer[b]), int(layer[d])) in _ALLOWED):
                tri.append((a, b, d))
    return np.asarray(tri, np.int64).reshape(-1, 3)


def link_labels(pid: np.ndarray, h0, h1, h2) -> np.ndarray:
    """Training label of a cell link: 1 if its three hits come from one particle."""
    pid = np.asarray(pid)
    p0, p1, p2 = pid[h0], pid[h1], pid[h2]
    return ((p0 >= 0) & (p0 == p1) & (p1 == p2)).astype(np.float32)


def match_fast(ntuplets: np.ndarray, pid: np.ndarray) -> np.ndarray:
    """Vectorised `match` with frac = 1: particle of each all-one-particle ntuplet, else -1."""
    nt = np.asarray(ntuplets)
    if nt.shape[0] == 0:
        return np.zeros(0, np.int64)
    valid = nt >= 0
    p = np.where(valid, np.asarray(pid)[np.where(valid, nt, 0)], -2)
    first = p[:, 0]
    same = np.all((p == first[:, None]) | ~valid, axis=1) & (first >= 0)
    return np.where(same, first, -1).astype(np.int64)


def rates_fast(ntuplets: np.ndarray, pid: np.ndarray, layer: np.ndarray,
               pairs=LAYER_PAIRS) -> dict:
    """`rates` with frac = 1, vectorised over ntuplets; reconstructable particles are
    those with a chain of >= 3 hits on `pairs`."""
    chains = particle_chains(pid, layer, pairs)
    reco = np.array([p for p, c in chains.items() if c["chain"].size >= 3], np.int64)
    m = match_fast(ntuplets, pid)
    matched, counts = np.unique(m[m >= 0], return_counts=True)
    hit = np.isin(reco, matched)
    cnt = dict(zip(matched.tolist(), counts.tolist()))
    dup = sum(1 for p in reco.tolist() if cnt.get(p, 0) > 1)
    n = max(reco.size, 1)
    return dict(efficiency=float(hit.sum()) / n, fake_rate=float(np.mean(m < 0)) if m.size else 0.0,
                duplicate_rate=dup / n, n_reconstructable=int(reco.size),
                n_ntuplets=int(m.size), n_fake=int(np.sum(m < 0)))
