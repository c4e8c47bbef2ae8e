"""Gate training checkpoints: the versioned binary round-trips bit-exactly and refuses
other files (CPU); a run interrupted and resumed from its checkpoint ends where an
uninterrupted run ends (GPU)."""

import os

import numpy as np
import pytest

from paper_2501_05520_gb300 import train_gate as tg


def _state(seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=tg.N_PARAMS).astype(np.float32) for _ in range(3)]


def test_checkpoint_round_trip(tmp_path):
    w, m, v = _state(1)
    p = str(tmp_path / "g.ckpt")
    tg.save_checkpoint(p, w, m, v, step=1234, epoch=2, pos=17, seed=5)
    ck = tg.load_checkpoint(p)
    for a, b in ((w, ck["w"]), (m, ck["m"]), (v, ck["v"])):
        assert a.tobytes() == b.tobytes()
    assert (ck["step"], ck["epoch"], ck["pos"], ck["seed"]) == (1234, 2, 17, 5)
    raw = open(p, "rb").read()
    assert raw[:4] == b"PTGC" and int.from_bytes(raw[4:8], "little") == tg.CKPT_VERSION
    assert len(raw) == 36 + 3 * 4 * tg.N_PARAMS
    assert not os.path.exists(p + ".tmp")


@pytest.mark.parametrize("damage", ["magic", "version", "short"])
def test_checkpoint_refuses_other_files(tmp_path, damage):
    p = str(tmp_path / "g.ckpt")
    tg.save_checkpoint(p, *_state(2), step=1, epoch=0, pos=1, seed=0)
    raw = bytearray(open(p, "rb").read())
    if damage == "magic":
        raw[0:4] = b"XXXX"
    elif damage == "version":
        raw[4:8] = (tg.CKPT_VERSION + 1).to_bytes(4, "little")
    else:
        raw = raw[:-4]
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        tg.load_checkpoint(p)


@pytest.mark.gpu
def test_interrupted_training_resumes(tmp_path):
    """64 Adam steps in one go, against 40 steps, a checkpoint, and the remaining 24 from
    it: the weights agree to 1e-4 relative (floor 1e-3).  The two runs take the same
    minibatches in the same order; what differs is only the order in which the gradient
    kernel's float32 atomics add up, which changes the last bits of each step."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    rng = np.random.default_rng(3)
    X = rng.normal(size=(32768, 12)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 3] > 0).astype(np.float32)
    kw = dict(epochs=2, batch=1024, lr=2e-3, seed=7, log=lambda *_: None)
    w_full = tg.train(X, y, **kw)
    ck = str(tmp_path / "g.ckpt")
    w_half = tg.train(X, y, checkpoint=ck, stop_after=40, **kw)
    assert tg.load_checkpoint(ck)["step"] == 40
    assert not np.allclose(w_half, w_full, rtol=1e-4, atol=1e-3)
    w_res = tg.train(X, y, checkpoint=ck, resume=True, **kw)
    assert np.allclose(w_res, w_full, rtol=1e-4, atol=1e-3)
    assert tg.load_checkpoint(ck)["step"] == 64
