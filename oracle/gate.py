"""CPU oracle of the learned link gate (TEST INFRASTRUCTURE ONLY).

Callers: the tests only (the training script runs the library's own kernels).  Shares
no code with the CUDA path.  Float64 throughout unless stated.

The gate is a small MLP that scores each accepted cell link (h0 -> h1 -> h2) and drops
links whose score is below a threshold before the ntuplet search.  It is the library's
analogue of the edge-filtering MLP of the paper's ML pipeline (Sec. 2.2.2: an MLP scores
graph edges and a fixed threshold removes clearly fake ones).  The paper gives no
architecture for this use; the library's reading is 12 -> 64 -> 64 -> 1 with ReLU,
BF16 weights and float32 accumulation on the GPU, a logit output, and binary
cross-entropy training on generator truth.

Parameter vector layout (5057 values): W1 [64,12], b1 [64], W2 [64,64], b2 [64],
w3 [64], b3 [1], row-major.

Features of a link (12), from the float32 hit coordinates (r = sqrt(x^2 + y^2)):
  0 C1 ratio |(z1-z0)(r2-r0) - (z2-z0)(r1-r0)| / (rz0 (r2-r0) + rz1 |z2-z0|)
  1 C2 ratio: curvature of the circle through the three hits / kmax
  2 C3 ratio: distance of closest approach of that circle to the z axis / dcamax(layer0)
  3 t_a / cotmax, t_a = (z1-z0)/(r1-r0)
  4 10 (t_b - t_a), t_b = (z2-z1)/(r2-r1)
  5..7 r0/16, r1/16, r2/16
  8 (z0 - r0 t_a) / z0max        (r-z line of the first cell at r = 0)
  9..11 layer0/9, layer1/9, layer2/9
"""

from __future__ import annotations

import numpy as np

N_FEAT = 12
HIDDEN = 64
N_PARAMS = HIDDEN * N_FEAT + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1  # 5057


def unpack(w: np.ndarray):
    w = np.asarray(w, np.float64)
    assert w.shape == (N_PARAMS,)
    o = 0
    W1 = w[o:o + HIDDEN * N_FEAT].reshape(HIDDEN, N_FEAT); o += HIDDEN * N_FEAT
    b1 = w[o:o + HIDDEN]; o += HIDDEN
    W2 = w[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = w[o:o + HIDDEN]; o += HIDDEN
    w3 = w[o:o + HIDDEN]; o += HIDDEN
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """He-style initialisation (float32 values)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / N_FEAT), (HIDDEN, N_FEAT))
    W2 = rng.normal(0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN))
    w3 = rng.normal(0, np.sqrt(1.0 / HIDDEN), HIDDEN)
    return pack(W1, np.zeros(HIDDEN), W2, np.zeros(HIDDEN), w3, 0.0).astype(np.float32)


def bf16_round(a) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(x, y, z, layer, h0, h1, h2, cuts: dict) -> np.ndarray:
    """Features [n, 12] of links given by hit index arrays, float64 from float32 hits."""
    x = np.asarray(x, np.float32).astype(np.float64)
    y = np.asarray(y, np.float32).astype(np.float64)
    z = np.asarray(z, np.float32).astype(np.float64)
    r = np.sqrt(x * x + y * y)
    p = [(x[h], y[h], z[h], r[h]) for h in (h0, h1, h2)]
    (x0, y0, z0, r0), (x1, y1, z1, r1), (x2, y2, z2, r2) = p
    c1 = np.abs((z1 - z0) * (r2 - r0) - (z2 - z0) * (r1 - r0)) / (
        cuts["rz0"] * (r2 - r0) + cuts["rz1"] * np.abs(z2 - z0))
    # circle through the three hits: curvature 2|A x B| / (|A| |B| |B - A|) with
    # A = P1 - P0, B = P2 - P0, and the distance of closest approach to the z axis
    # | |C| - R | written without dividing by A x B (finite for collinear hits, where it
    # is the distance of the line)
    ax, ay, bx, by = x1 - x0, y1 - y0, x2 - x0, y2 - y0
    a2, b2 = ax * ax + ay * ay, bx * bx + by * by
    cr = ax * by - ay * bx
    kappa = 2.0 * np.abs(cr) / (np.sqrt(a2) * np.sqrt(b2) * np.hypot(x2 - x1, y2 - y1))
    D = 2.0 * cr
    ux, uy = by * a2 - ay * b2, ax * b2 - bx * a2
    num = (x0 * x0 + y0 * y0) * D + 2.0 * (x0 * ux + y0 * uy)
    den = np.hypot(x0 * D + ux, y0 * D + uy) + np.hypot(ux, uy)
    dca = np.abs(num) / den
    dmax = np.where(np.asarray(layer)[h0] == 0, cuts["dca_b0"], cuts["dca_other"])
    ta = (z1 - z0) / (r1 - r0)
    tb = (z2 - z1) / (r2 - r1)
    L = np.asarray(layer).astype(np.float64)
    return np.stack([c1, kappa / cuts["kmax"], dca / dmax, ta / cuts["cotmax"], 10.0 * (tb - ta),
                     r0 / 16.0, r1 / 16.0, r2 / 16.0, (z0 - r0 * ta) / cuts["z0max"],
                     L[h0] / 9.0, L[h1] / 9.0, L[h2] / 9.0], axis=1)


def forward(w, X, bf16: bool = False):
    """Logits [n].  bf16: weights, inputs and the hidden activations fed to the next
    layer are rounded to bfloat16 (what the tensor-core inference consumes); the sums
    are exact (float64)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    if bf16:
        W1, W2 = bf16_round(W1), bf16_round(W2)
        X = bf16_round(X.astype(np.float32))
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    if bf16:
        h1 = bf16_round(h1.astype(np.float32))
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(w, X, y):
    """Mean binary cross-entropy of sigmoid(logit) against labels y, and its gradient
    with respect to the 5057 parameters (float64 backpropagation)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w3 + b3
    # stable BCE: log(1 + exp(s)) - y s
    loss = np.mean(np.logaddexp(0.0, s) - y * s)
    ds = (1.0 / (1.0 + np.exp(-s)) - y) / n
    gw3 = h2.T @ ds
    gb3 = ds.sum()
    dz2 = np.outer(ds, w3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def link_labels(pid, h0, h1, h2) -> np.ndarray:
    """1 where the three hits come from one generated particle, else 0."""
    pid = np.asarray(pid)
    p0, p1, p2 = pid[h0], pid[h1], pid[h2]
    return ((p0 >= 0) & (p0 == p1) & (p1 == p2)).astype(np.float32)
