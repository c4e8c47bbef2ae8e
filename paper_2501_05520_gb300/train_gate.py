"""Training of the learned link gate on the GPU with the library's own kernels.

  python -m paper_2501_05520_gb300.train_gate --out gate.npz

Data: every link the plain cellular automaton accepts on N synthetic PU200 events
(seeds 4_000_000 + i, disjoint from the evaluation seeds), with its 12 features from
pt_get_link_features and a generator-truth label (1 if the three hits belong to one
particle, sim.truth.link_labels).  Training: mean binary cross-entropy, Adam on
minibatches, every loss/gradient/update computed by pt_gate_loss_grad and
pt_gate_adam (torch holds the device buffers only).  Threshold: the largest tau that
keeps a target fraction of the true links of a validation split (seeds
4_100_000 + i), scored by the tensor-core inference path (pt_gate_score).
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import paper_2501_05520_gb300 as pt  # noqa: E402
import sim  # noqa: E402
from sim import truth  # noqa: E402

N_PARAMS = 5057
TRAIN_SEED0 = 4_000_000
VAL_SEED0 = 4_100_000


def init_params(seed: int) -> np.ndarray:
    """He initialisation of W1, W2, w3; zero biases (parameter layout of pt_set_gate)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / 12), (64, 12))
    W2 = rng.normal(0, np.sqrt(2.0 / 64), (64, 64))
    w3 = rng.normal(0, np.sqrt(1.0 / 64), 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]]
                          ).astype(np.float32)


def link_dataset(n_events: int, seed0: int, cuts: dict, ctx) -> tuple[np.ndarray, np.ndarray]:
    """Features and labels of all plain-CA links of n_events PU200 events."""
    xs, ys = [], []
    for i in range(n_events):
        ev = sim.generate(sim.PU200, seed0 + i)
        ctx.pt_load_hits(ev.x, ev.y, ev.z, ev.layer)
        ctx.pt_build_doublets(sync=False)
        ctx.pt_connect_cells()
        feat, h0, h1, h2, _, _ = ctx.pt_get_link_features()
        xs.append(feat)
        ys.append(truth.link_labels(ev.pid, h0, h1, h2))
    return np.concatenate(xs), np.concatenate(ys)


def train(X: np.ndarray, y: np.ndarray, epochs: int = 4, batch: int = 4096, lr: float = 2e-3,
          seed: int = 0, log=print) -> np.ndarray:
    import torch
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    dX = torch.from_numpy(X[perm]).cuda()
    dy = torch.from_numpy(y[perm]).cuda()
    w = torch.from_numpy(init_params(seed)).cuda()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    grad = torch.empty_like(w)
    loss = torch.empty(1, device="cuda")
    nb = X.shape[0] // batch
    step = 0
    for ep in range(epochs):
        lr_ep = lr if ep < epochs - 1 else lr * 0.25
        acc = torch.zeros(1, device="cuda")
        for bi in rng.permutation(nb):
            sl = slice(int(bi) * batch, (int(bi) + 1) * batch)
            pt.pt_gate_loss_grad(w, dX[sl], dy[sl], grad, loss)
            step += 1
            pt.pt_gate_adam(w, m, v, grad, lr_ep, step)
            acc += loss
        log(f"epoch {ep}: mean loss {float(acc.item()) / max(nb, 1):.4f} ({step} steps)")
    return w.cpu().numpy()


def choose_tau(w: np.ndarray, X: np.ndarray, y: np.ndarray, keep_true: float, ctx) -> float:
    """Largest threshold keeping `keep_true` of the true links (tensor-core scores)."""
    import torch
    ctx.pt_set_gate(w, 0.0)
    chunk = int(ctx.capacity["max_links"])
    s = np.empty(X.shape[0], np.float32)
    for i in range(0, X.shape[0], chunk):
        d = torch.from_numpy(X[i:i + chunk]).cuda()
        out = torch.empty(d.shape[0], device="cuda")
        ctx.pt_gate_score(d, out)
        s[i:i + chunk] = out.cpu().numpy()
    ctx.pt_set_gate(None, 0.0)
    return float(np.quantile(s[y > 0.5], 1.0 - keep_true))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train-events", type=int, default=200)
    ap.add_argument("--val-events", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--keep-true", type=float, default=0.998)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    from paper_2501_05520_gb300 import build
    build.build()
    cuts = pt.default_cuts()
    cap = pt.default_capacity(max_events=1, hits_per_event=65536, cells_per_event=4 << 20,
                              links_per_event=1 << 20, ntuplets_per_event=1 << 19)
    t0 = time.time()
    with pt.Context(cuts=cuts, capacity=cap) as ctx:
        X, y = link_dataset(a.train_events, TRAIN_SEED0, cuts, ctx)
        Xv, yv = link_dataset(a.val_events, VAL_SEED0, cuts, ctx)
        print(f"dataset: {X.shape[0]} training links ({y.mean():.3f} true), {Xv.shape[0]} "
              f"validation, {time.time() - t0:.1f} s")
        t1 = time.time()
        w = train(X, y, epochs=a.epochs, seed=a.seed)
        print(f"training: {time.time() - t1:.1f} s")
        tau = choose_tau(w, Xv, yv, a.keep_true, ctx)
    meta = dict(train_seeds=[TRAIN_SEED0, TRAIN_SEED0 + a.train_events],
                val_seeds=[VAL_SEED0, VAL_SEED0 + a.val_events], epochs=a.epochs,
                keep_true=a.keep_true, n_train=int(X.shape[0]), seed=a.seed,
                command="python -m paper_2501_05520_gb300.train_gate " + " ".join(argv or sys.argv[1:]))
    np.savez(a.out, w=w.astype(np.float32), tau=np.float32(tau), meta=json.dumps(meta))
    print(f"tau = {tau:.4f}; saved {a.out}")


if __name__ == "__main__":
    main()
