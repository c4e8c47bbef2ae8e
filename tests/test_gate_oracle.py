"""Pins of the gate oracle (oracle/gate.py): backpropagation against central finite
differences, a hand-computable forward pass, bfloat16 rounding against its definition,
and link features against independent geometry on the oracle's own links."""

import math

import numpy as np
import pytest

import oracle
import sim
from oracle import gate


def test_param_count():
    assert gate.N_PARAMS == 5057


def test_bf16_round_definition():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-3, 65504.0], np.float32)
    got = gate.bf16_round(vals)
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-9 rounds up
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -7
    assert got[3] == -2.5
    for v, g in zip(vals, got):
        assert abs(g - v) <= 2 ** -8 * abs(v) + 1e-45  # half an ulp, 8-bit significand


def test_forward_hand_computed():
    W1 = np.zeros((64, 12)); W1[0, 0] = 2.0; W1[1, 1] = -1.0
    b1 = np.zeros(64); b1[1] = 0.5
    W2 = np.zeros((64, 64)); W2[0, 0] = 1.0; W2[0, 1] = 3.0
    b2 = np.zeros(64)
    w3 = np.zeros(64); w3[0] = 0.25
    w = gate.pack(W1, b1, W2, b2, w3, -1.0)
    X = np.zeros((2, 12)); X[0, 0] = 1.0; X[1, 1] = 0.25
    # h1 = relu(2 x0, 0.5 - x1); h2_0 = h1_0 + 3 h1_1; s = 0.25 h2_0 - 1
    exp = [0.25 * (2.0 + 3 * 0.5) - 1.0, 0.25 * (3 * 0.25) - 1.0]
    assert np.allclose(gate.forward(w, X), exp, rtol=0, atol=1e-15)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = gate.init_params(5).astype(np.float64)
    w[gate.N_PARAMS - 1] = 0.1
    X = rng.normal(0, 1, (64, 12))
    y = (rng.random(64) < 0.5).astype(np.float64)
    loss, g = gate.loss_and_grad(w, X, y)
    eps = 1e-6
    idx = rng.choice(gate.N_PARAMS, 200, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd = (gate.loss_and_grad(wp, X, y)[0] - gate.loss_and_grad(wm, X, y)[0]) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i
    # loss is the BCE of the forward logits
    s = gate.forward(w, X)
    assert loss == pytest.approx(np.mean(np.log1p(np.exp(-s)) * y + np.log1p(np.exp(s)) * (1 - y)))


def _circle(p0, p1, p2):
    A = 2.0 * np.array([p1 - p0, p2 - p0])
    b = np.array([p1 @ p1 - p0 @ p0, p2 @ p2 - p0 @ p0])
    c = np.linalg.solve(A, b)
    return c, float(np.hypot(*(p0 - c)))


def test_features_on_oracle_links(cuts):
    ev = sim.generate(sim.PU50, 2300, n_particles=300)
    res = oracle.reconstruct(ev.x, ev.y, ev.z, ev.layer, cuts)
    ci, co = res["cell_inner"], res["cell_outer"]
    h0, h1, h2 = ci[res["link_a"]], co[res["link_a"]], co[res["link_b"]]
    F = gate.features(ev.x, ev.y, ev.z, ev.layer, h0, h1, h2, cuts)
    assert F.shape == (h0.size, 12) and h0.size > 100
    # accepted links pass every cut, so the three cut ratios are <= 1
    assert np.all(F[:, :3] <= 1.0 + 1e-5)
    # the C3 ratio equals the link quality over its threshold
    dmax = np.where(ev.layer[h0] == 0, cuts["dca_b0"], cuts["dca_other"])
    # (the float32 link quality carries cancellation error for small distances)
    assert np.allclose(F[:, 2], res["link_q"] / dmax, rtol=1e-4, atol=2e-4)
    x, y = ev.x.astype(np.float64), ev.y.astype(np.float64)
    for k in range(0, h0.size, 7):
        P = [np.array([x[h], y[h]]) for h in (h0[k], h1[k], h2[k])]
        c, R = _circle(*P)
        assert F[k, 1] * cuts["kmax"] == pytest.approx(1.0 / R, rel=1e-6)
        assert F[k, 2] * dmax[k] == pytest.approx(abs(math.hypot(*c) - R), rel=1e-4, abs=1e-7)
    assert np.all((F[:, 9:] >= 0) & (F[:, 9:] <= 1))
