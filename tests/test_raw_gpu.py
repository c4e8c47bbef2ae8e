"""GPU parity of raw pixel data -> hits (pt_set_modules / pt_load_raw / pt_get_hits)
against the float64 oracle (oracle/pixels.py), and the chain fed from raw data.

Hits must come in the oracle's order with the same layers; positions within 2e-5 cm
(float32 azimuth, radius and sine/cosine against float64: a few 1e-7 relative of
coordinates up to 52 cm).  The chain run on the raw-made hits must give the same
ntuplets as the chain run on the same hits loaded with pt_load_batch.
"""

import numpy as np
import pytest

import sim
from oracle import pixels as opix
from sim import pixels as simpix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2501_05520_gb300 as pt  # noqa: E402
from paper_2501_05520_gb300 import pixels as ppix  # noqa: E402

CAP = pt.default_capacity(max_events=6, hits_per_event=65536, cells_per_event=4 << 20,
                          links_per_event=1 << 20, ntuplets_per_event=1 << 19)
TOL = 2e-5


@pytest.fixture(scope="module")
def raw_batch():
    empty = sim.generate(sim.PU50, 2001)
    for f in ("x", "y", "z", "layer", "pid", "x64", "y64", "z64"):
        setattr(empty, f, getattr(empty, f)[:0])
    events = [sim.generate(sim.PU50, 2000), empty,
              sim.generate(sim.SINGLE_MUON_LIKE, 1007, n_particles=2),
              sim.generate(sim.PU200, 3100)]
    raws = [simpix.digitize(ev)[0] for ev in events]
    return events, raws


def test_raw_hits_match_oracle(cuts, raw_batch):
    events, raws = raw_batch
    table = opix.modules(ppix.PARAMS)
    off, words = simpix.concat_raw(raws)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_modules()
        nh = ctx.pt_load_raw(off, words)
        x, y, z, layer, hoff = ctx.pt_get_hits()
        # the chain on these hits, fed from raw data and again as ordinary inputs
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_find_ntuplets()
        ctx.pt_fit_tracks()
        nt_raw, _, ev_raw = ctx.pt_get_ntuplets()
        tr_raw = ctx.pt_get_tracks()
        ctx.pt_load_batch(hoff, x, y, z, layer)
        ctx.pt_build_doublets()
        ctx.pt_connect_cells()
        ctx.pt_find_ntuplets()
        ctx.pt_fit_tracks()
        nt_std, _, ev_std = ctx.pt_get_ntuplets()
        tr_std = ctx.pt_get_tracks()
    assert nh == x.size and hoff[0] == 0 and hoff[-1] == nh
    for e, w in enumerate(raws):
        rx, ry, rz, rl, _ = opix.reconstruct(w, table)
        sl = slice(hoff[e], hoff[e + 1])
        assert hoff[e + 1] - hoff[e] == rx.size
        np.testing.assert_array_equal(layer[sl], rl.astype(np.uint8))
        for got, exp in ((x[sl], rx), (y[sl], ry), (z[sl], rz)):
            assert np.max(np.abs(got.astype(np.float64) - exp), initial=0.0) <= TOL
    assert ev_raw.tolist() == ev_std.tolist()
    assert np.array_equal(nt_raw, nt_std)
    assert tr_raw.tobytes() == tr_std.tobytes()
    assert nt_raw.shape[0] > 1000


def _words(module, pixels):
    return np.asarray([(module << 40) | (r << 28) | (c << 16) | a for r, c, a in pixels], np.uint64)


def test_raw_input_errors(cuts):
    good = _words(5, [(3, 3, 50), (3, 4, 60)])
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        with pytest.raises(pt.PtError) as err:  # no module table yet
            ctx.pt_load_raw([0, 2], good)
        assert err.value.status == pt.PT_ERR_INVALID
        ctx.pt_set_modules()
        assert ctx.pt_load_raw([0, 2], good) == 1
        bad = {
            "module outside the table": _words(1 << 20, [(0, 0, 9)]),
            "row outside the module": _words(5, [(4000, 0, 9)]),
            "adc above 4095": _words(5, [(0, 0, 5000)]),
            "pixels out of order": _words(5, [(3, 4, 9), (3, 3, 9)]),
            "pixel twice": _words(5, [(3, 3, 9), (3, 3, 9)]),
        }
        for why, w in bad.items():
            with pytest.raises(pt.PtError) as err:
                ctx.pt_load_raw([0, w.size], w)
            assert err.value.status == pt.PT_ERR_INVALID, why
        many = _words(5, [(r, c, 9) for r in range(11) for c in range(100)])  # 1100 digis
        with pytest.raises(pt.PtError) as err:
            ctx.pt_load_raw([0, many.size], many)
        assert err.value.status == pt.PT_ERR_CAPACITY
        big = _words(5, [(r, c, 9) for r in range(12) for c in range(12)])  # 144-pixel cluster
        with pytest.raises(pt.PtError) as err:
            ctx.pt_load_raw([0, big.size], big)
        assert err.value.status == pt.PT_ERR_CAPACITY
        # the same errors inside runs long enough for the block-per-run launch
        grid = [(r, c, 9) for r in range(0, 60, 3) for c in range(0, 45, 3)]  # 300 isolated
        long_bad = _words(5, grid[:150] + [(200, 1, 9), (199, 1, 9)] + grid[152:])
        assert long_bad.size == 300
        with pytest.raises(pt.PtError) as err:
            ctx.pt_load_raw([0, long_bad.size], long_bad)
        assert err.value.status == pt.PT_ERR_INVALID
        blob = [(r, c, 9) for r in range(100, 112) for c in range(0, 12)]  # 144 pixels
        long_big = _words(5, sorted(grid[:200] + blob))
        with pytest.raises(pt.PtError) as err:
            ctx.pt_load_raw([0, long_big.size], long_big)
        assert err.value.status == pt.PT_ERR_CAPACITY
        with pytest.raises(ValueError):
            ctx.pt_load_raw([0, 3], good)  # offsets beyond the digis given
        # a valid batch after the errors works again
        assert ctx.pt_load_raw([0, 2, 2], good) == 1


def _sparse_run(rng, module, n, nrow, ncol):
    """n distinct pixels of one module in (row, col) order, sparse enough that clusters
    stay small."""
    flat = np.sort(rng.choice(nrow * ncol, size=n, replace=False))
    adc = rng.integers(5, 4096, size=n)
    return _words(module, [(int(f // ncol), int(f % ncol), int(a)) for f, a in zip(flat, adc)])


@pytest.mark.parametrize("sizes", [(1, 255, 256, 257), (1024, 300, 2)])
def test_raw_run_sizes(cuts, sizes):
    """Runs on both sides of the warp-per-run / block-per-run split and at the largest
    size a run may have, against the oracle."""
    table = opix.modules(ppix.PARAMS)
    rng = np.random.default_rng(sum(sizes))
    mods = [3, 40, 500, 1000]
    ev = np.concatenate([_sparse_run(rng, m, n, int(table[m, 8]), int(table[m, 7]))
                         for m, n in zip(mods, sizes)])
    raws = [ev, ev[: sizes[0]]]
    off, words = simpix.concat_raw(raws)
    with pt.Context(cuts=cuts, capacity=CAP) as ctx:
        ctx.pt_set_modules()
        ctx.pt_load_raw(off, words)
        x, y, z, layer, hoff = ctx.pt_get_hits()
    for e, w in enumerate(raws):
        rx, ry, rz, rl, _ = opix.reconstruct(w, table)
        sl = slice(hoff[e], hoff[e + 1])
        assert hoff[e + 1] - hoff[e] == rx.size
        np.testing.assert_array_equal(layer[sl], rl.astype(np.uint8))
        for got, exp in ((x[sl], rx), (y[sl], ry), (z[sl], rz)):
            assert np.max(np.abs(got.astype(np.float64) - exp), initial=0.0) <= TOL
