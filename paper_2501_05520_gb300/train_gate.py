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

Checkpoints (--checkpoint PATH, written every --checkpoint-every steps and at the end;
--resume continues from one): a versioned little-endian binary holding the weights, the
Adam moments m and v, the step count and the position in the minibatch order, so that an
interrupted run resumes where it stopped with the same minibatches and optimiser state.
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

# Checkpoint layout, little-endian: a 36-byte header (magic b"PTGC", u32 version,
# u32 n_params, u64 step, u32 epoch, u32 position in that epoch's minibatch order, u64
# data seed), then float32 w, m, v (n_params each).
CKPT_MAGIC = b"PTGC"
CKPT_VERSION = 1
_CKPT_HEAD = np.dtype([("magic", "S4"), ("version", "<u4"), ("n", "<u4"), ("step", "<u8"),
                       ("epoch", "<u4"), ("pos", "<u4"), ("seed", "<u8")])


def save_checkpoint(path: str, w, m, v, step: int, epoch: int, pos: int, seed: int) -> None:
    """Writes the training state (atomically: a temporary file renamed over `path`)."""
    head = np.zeros(1, _CKPT_HEAD)
    head[0] = (CKPT_MAGIC, CKPT_VERSION, N_PARAMS, step, epoch, pos, seed)
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(head.tobytes())
        for a in (w, m, v):
            a = np.asarray(a, np.float32)
            if a.shape != (N_PARAMS,):
                raise ValueError("checkpoint arrays must hold N_PARAMS float32 values")
            f.write(a.astype("<f4").tobytes())
    os.replace(tmp, path)


def load_checkpoint(path: str) -> dict:
    """Reads a checkpoint; ValueError on a wrong magic, version, size or length."""
    raw = open(path, "rb").read()
    if len(raw) != _CKPT_HEAD.itemsize + 3 * 4 * N_PARAMS:
        raise ValueError(f"{path}: {len(raw)} bytes, not a gate checkpoint")
    head = np.frombuffer(raw[:_CKPT_HEAD.itemsize], _CKPT_HEAD)[0]
    if head["magic"] != CKPT_MAGIC or int(head["version"]) != CKPT_VERSION or \
            int(head["n"]) != N_PARAMS:
        raise ValueError(f"{path}: not a version-{CKPT_VERSION} gate checkpoint")
    arr = np.frombuffer(raw[_CKPT_HEAD.itemsize:], "<f4").reshape(3, N_PARAMS).astype(np.float32)
    return dict(w=arr[0], m=arr[1], v=arr[2], step=int(head["step"]), epoch=int(head["epoch"]),
                pos=int(head["pos"]), seed=int(head["seed"]))


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
          seed: int = 0, log=print, checkpoint: str | None = None, checkpoint_every: int = 0,
          resume: bool = False, stop_after: int | None = None) -> np.ndarray:
    """Adam on minibatches of (X, y).  The example order and every epoch's minibatch order
    come from one generator seeded with `seed`, so a run resumed from a checkpoint takes
    the same minibatches as an uninterrupted one.  stop_after: end (writing the
    checkpoint) after that many steps in total, as an interrupted run would."""
    import torch
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    dX = torch.from_numpy(X[perm]).cuda()
    dy = torch.from_numpy(y[perm]).cuda()
    nb = X.shape[0] // batch
    orders = [rng.permutation(nb) for _ in range(epochs)]
    w = torch.from_numpy(init_params(seed)).cuda()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    step, ep0, pos0 = 0, 0, 0
    if resume:
        ck = load_checkpoint(checkpoint)
        if ck["seed"] != seed:
            raise ValueError("the checkpoint was written by a run with another seed")
        for dst, src in ((w, ck["w"]), (m, ck["m"]), (v, ck["v"])):
            dst.copy_(torch.from_numpy(src))
        step, ep0, pos0 = ck["step"], ck["epoch"], ck["pos"]
        log(f"resumed at step {step} (epoch {ep0}, minibatch {pos0})")
    grad = torch.empty_like(w)
    loss = torch.empty(1, device="cuda")

    def save(ep, pos):
        if checkpoint:
            save_checkpoint(checkpoint, w.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), step,
                            ep, pos, seed)

    for ep in range(ep0, epochs):
        lr_ep = lr if ep < epochs - 1 else lr * 0.25
        acc = torch.zeros(1, device="cuda")
        for pos in range(pos0 if ep == ep0 else 0, nb):
            if stop_after is not None and step >= stop_after:
                save(ep, pos)
                return w.cpu().numpy()
            bi = int(orders[ep][pos])
            sl = slice(bi * batch, (bi + 1) * batch)
            pt.pt_gate_loss_grad(w, dX[sl], dy[sl], grad, loss)
            step += 1
            pt.pt_gate_adam(w, m, v, grad, lr_ep, step)
            acc += loss
            if checkpoint_every and step % checkpoint_every == 0:
                save(ep, pos + 1)
        log(f"epoch {ep}: mean loss {float(acc.item()) / max(nb, 1):.4f} ({step} steps)")
    save(epochs, 0)
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
    ap.add_argument("--checkpoint", default=None, help="training-state file (written)")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
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
        w = train(X, y, epochs=a.epochs, seed=a.seed, checkpoint=a.checkpoint,
                  checkpoint_every=a.checkpoint_every if a.checkpoint else 0,
                  resume=a.resume)
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
