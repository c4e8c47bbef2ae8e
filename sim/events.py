"""Seeded synthetic pixel events: charged helices in a solenoid, plus uniform noise.

This module is the input recipe shared by the tests, the benchmark and the training
driver.  It contains no reconstruction arithmetic: it draws particles, intersects
their helices with the detector surfaces and smears the crossings.

Units: cm, GeV, tesla.  Magnetic field along +z.

Detector (layer codes are part of the library's input contract):
  0..3  barrel cylinders, r = 2.9 / 6.8 / 10.9 / 16.0 cm, |z| < 27 cm
  4..6  disks at z = +29.1 / +39.6 / +51.6 cm, 4.5 <= r <= 16 cm
  7..9  disks at z = -29.1 / -39.6 / -51.6 cm, same radial extent

The paper's workloads are CMS HLT data and ACTS ttbar events at pileup 200
(Sec. 2.2.2); neither is available, so these helices stand in for them.
"""

from __future__ import annotations

import dataclasses
import numpy as np

BFIELD_T = 3.8
# GeV per (T * m): pT = C_LIGHT * B * R[m]
C_LIGHT = 0.299792458

BARREL_R = (2.9, 6.8, 10.9, 16.0)
BARREL_ZMAX = 27.0
DISK_Z = (29.1, 39.6, 51.6)
DISK_RMIN = 4.5
DISK_RMAX = 16.0
N_LAYERS = 10

SIGMA_RPHI = 10e-4  # 10 um
SIGMA_Z = 20e-4     # 20 um (barrel z, disk r)


def layer_surface(layer: int):
    """Return ('barrel', r) or ('disk', z) for a layer code."""
    if layer < 4:
        return "barrel", BARREL_R[layer]
    if layer < 7:
        return "disk", DISK_Z[layer - 4]
    return "disk", -DISK_Z[layer - 7]


@dataclasses.dataclass
class Event:
    """One synthetic event, hits in a random order.

    x, y, z : float32 hit coordinates (what the library receives)
    layer   : uint8 layer codes
    pid     : int32 generating particle per hit, -1 for noise
    x64,y64,z64 : float64 coordinates before the float32 rounding (after smearing)
    xt,yt,zt    : float64 noiseless crossings (NaN for noise hits)
    particles   : dict of per-particle float64 arrays (pt, eta, phi0, z0, q, R)
    seed        : generator seed
    """

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    layer: np.ndarray
    pid: np.ndarray
    x64: np.ndarray
    y64: np.ndarray
    z64: np.ndarray
    xt: np.ndarray
    yt: np.ndarray
    zt: np.ndarray
    particles: dict
    seed: int

    @property
    def n_hits(self) -> int:
        return int(self.x.shape[0])


@dataclasses.dataclass(frozen=True)
class GenConfig:
    n_particles: int
    spectrum: str          # "inv_pt_uniform" (1/pT ~ U[0.1, 2]) or "exp" (0.3 + Exp(1))
    eta_max: float
    barrel_only: bool
    noise_frac: float
    z0_sigma: float = 5.0
    smear: bool = True


# The five workloads.  Sizes and spectra follow the library's benchmark definitions.
SINGLE_MUON_LIKE = GenConfig(50, "inv_pt_uniform", 1.0, True, 0.0)          # ~200 hits
PU50 = GenConfig(2500, "exp", 2.5, False, 0.01)                              # ~12k hits
PU200 = GenConfig(10000, "inv_pt_uniform", 2.5, False, 0.02)                 # ~50k hits
PARTICLES_PER_PU = 50


def _draw_particles(rng: np.random.Generator, cfg: GenConfig, n: int) -> dict:
    if cfg.spectrum == "inv_pt_uniform":
        pt = 1.0 / rng.uniform(0.1, 2.0, n)
    elif cfg.spectrum == "exp":
        pt = 0.3 + rng.exponential(1.0, n)
    else:
        raise ValueError(cfg.spectrum)
    eta = rng.uniform(-cfg.eta_max, cfg.eta_max, n)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    z0 = rng.normal(0.0, cfg.z0_sigma, n)
    R = pt / (C_LIGHT * BFIELD_T) * 100.0
    return dict(pt=pt, eta=eta, phi0=phi0, q=q, z0=z0, R=R)


def _crossings(p: dict, barrel_only: bool):
    """Noiseless helix/surface crossings.  Returns (pid, layer, x, y, z) float64 arrays."""
    n = p["pt"].shape[0]
    ids = np.arange(n)
    sh = np.sinh(p["eta"])
    out = []
    for L, rl in enumerate(BARREL_R):
        ok = rl < 2.0 * p["R"]
        arg = np.where(ok, rl / (2.0 * p["R"]), 0.0)
        alpha = 2.0 * np.arcsin(arg)
        s = p["R"] * alpha
        z = p["z0"] + s * sh
        keep = ok & (np.abs(z) < BARREL_ZMAX)
        phi = p["phi0"] - p["q"] * alpha / 2.0
        out.append((ids[keep], np.full(keep.sum(), L), rl * np.cos(phi[keep]),
                    rl * np.sin(phi[keep]), z[keep]))
    if not barrel_only:
        for side in (+1, -1):
            for k, zd_abs in enumerate(DISK_Z):
                zd = side * zd_abs
                L = 4 + k if side > 0 else 7 + k
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = (zd - p["z0"]) / sh
                alpha = s / p["R"]
                ok = np.isfinite(s) & (s > 0) & (alpha < np.pi)
                alpha = np.where(ok, alpha, 0.0)
                r = 2.0 * p["R"] * np.sin(alpha / 2.0)
                keep = ok & (r >= DISK_RMIN) & (r <= DISK_RMAX)
                phi = p["phi0"] - p["q"] * alpha / 2.0
                out.append((ids[keep], np.full(keep.sum(), L), r[keep] * np.cos(phi[keep]),
                            r[keep] * np.sin(phi[keep]), np.full(keep.sum(), zd)))
    pid = np.concatenate([o[0] for o in out]).astype(np.int32)
    lay = np.concatenate([o[1] for o in out]).astype(np.uint8)
    x = np.concatenate([o[2] for o in out])
    y = np.concatenate([o[3] for o in out])
    z = np.concatenate([o[4] for o in out])
    return pid, lay, x, y, z


def _smear(rng, lay, x, y, z):
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    barrel = lay < 4
    n = x.shape[0]
    g1 = rng.normal(0.0, 1.0, n)
    g2 = rng.normal(0.0, 1.0, n)
    phi = phi + g1 * SIGMA_RPHI / r
    r_new = np.where(barrel, r, r + g2 * SIGMA_Z)
    z_new = np.where(barrel, z + g2 * SIGMA_Z, z)
    return r_new * np.cos(phi), r_new * np.sin(phi), z_new


def _noise(rng, n_noise: int, barrel_only: bool):
    areas = [2.0 * np.pi * rl * 2.0 * BARREL_ZMAX for rl in BARREL_R]
    layers = list(range(4))
    if not barrel_only:
        a_disk = np.pi * (DISK_RMAX**2 - DISK_RMIN**2)
        areas += [a_disk] * 6
        layers += list(range(4, 10))
    areas = np.asarray(areas)
    lay = rng.choice(np.asarray(layers), size=n_noise, p=areas / areas.sum()).astype(np.uint8)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_noise)
    u = rng.random(n_noise)
    x = np.empty(n_noise)
    y = np.empty(n_noise)
    z = np.empty(n_noise)
    for L in np.unique(lay):
        m = lay == L
        kind, v = layer_surface(int(L))
        if kind == "barrel":
            r = np.full(m.sum(), v)
            z[m] = -BARREL_ZMAX + 2.0 * BARREL_ZMAX * u[m]
        else:
            r = np.sqrt(DISK_RMIN**2 + (DISK_RMAX**2 - DISK_RMIN**2) * u[m])
            z[m] = v
        x[m] = r * np.cos(phi[m])
        y[m] = r * np.sin(phi[m])
    return lay, x, y, z


def generate(cfg: GenConfig, seed: int, n_particles: int | None = None,
             n_vertices: int = 0) -> Event:
    """Generate one event from a seed.  Hits are returned in a random order.

    n_vertices > 0 groups the particles into that many interactions of equal size
    (particle i belongs to vertex i * n_vertices // n): each vertex draws its z from
    N(0, cfg.z0_sigma) and its particles share it; particles["vertex"] and
    particles["vz"] record the assignment.  With n_vertices = 0 (the default) every
    particle draws its own z0 and the event is unchanged."""
    rng = np.random.default_rng(seed)
    n = cfg.n_particles if n_particles is None else n_particles
    p = _draw_particles(rng, cfg, n)
    if n_vertices > 0:
        vz = rng.normal(0.0, cfg.z0_sigma, n_vertices)
        vid = (np.arange(n) * n_vertices) // max(n, 1)
        p["z0"] = vz[vid]
        p["vertex"] = vid.astype(np.int32)
        p["vz"] = vz
    pid, lay, xt, yt, zt = _crossings(p, cfg.barrel_only)
    if cfg.smear:
        xs, ys, zs = _smear(rng, lay, xt, yt, zt)
    else:
        xs, ys, zs = xt.copy(), yt.copy(), zt.copy()
    n_noise = int(round(cfg.noise_frac * pid.shape[0]))
    if n_noise:
        nl, nx, ny, nz = _noise(rng, n_noise, cfg.barrel_only)
        pid = np.concatenate([pid, np.full(n_noise, -1, np.int32)])
        lay = np.concatenate([lay, nl])
        xs = np.concatenate([xs, nx])
        ys = np.concatenate([ys, ny])
        zs = np.concatenate([zs, nz])
        nan = np.full(n_noise, np.nan)
        xt = np.concatenate([xt, nan])
        yt = np.concatenate([yt, nan])
        zt = np.concatenate([zt, nan])
    order = rng.permutation(pid.shape[0])
    return Event(
        x=xs[order].astype(np.float32), y=ys[order].astype(np.float32),
        z=zs[order].astype(np.float32), layer=lay[order].astype(np.uint8),
        pid=pid[order].astype(np.int32),
        x64=xs[order], y64=ys[order], z64=zs[order],
        xt=xt[order], yt=yt[order], zt=zt[order], particles=p, seed=seed)


def single_helix(seed: int, pt: float, eta: float, phi0: float, q: float, z0: float,
                 barrel_only: bool = True) -> Event:
    """One noiseless particle with the given parameters (no smearing)."""
    p = dict(pt=np.array([pt]), eta=np.array([eta]), phi0=np.array([phi0]),
             q=np.array([q]), z0=np.array([z0]),
             R=np.array([pt / (C_LIGHT * BFIELD_T) * 100.0]))
    pid, lay, xt, yt, zt = _crossings(p, barrel_only)
    rng = np.random.default_rng(seed)
    order = rng.permutation(pid.shape[0])
    return Event(
        x=xt[order].astype(np.float32), y=yt[order].astype(np.float32),
        z=zt[order].astype(np.float32), layer=lay[order], pid=pid[order],
        x64=xt[order], y64=yt[order], z64=zt[order],
        xt=xt[order], yt=yt[order], zt=zt[order], particles=p, seed=seed)


def pileup_event(seed: int, pu: int, noise_frac: float = 0.02) -> Event:
    """PU200-spectrum event with `pu` * 50 particles (batch and serving workloads)."""
    cfg = dataclasses.replace(PU200, noise_frac=noise_frac)
    return generate(cfg, seed, n_particles=pu * PARTICLES_PER_PU)


def vertex_event(seed: int, pu: int, noise_frac: float = 0.02, smear: bool = True) -> Event:
    """PU200-spectrum event with `pu` interactions of 50 particles each, every
    interaction at its own z ~ N(0, 5 cm) (vertex reconstruction workload)."""
    cfg = dataclasses.replace(PU200, noise_frac=noise_frac, smear=smear)
    return generate(cfg, seed, n_particles=pu * PARTICLES_PER_PU, n_vertices=pu)


def batch_pileups(seed: int, n_events: int = 64, mean: float = 140.0,
                  lo: int = 20, hi: int = 250) -> np.ndarray:
    """Per-event pileup for the batched workload: Poisson(mean) clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.clip(rng.poisson(mean, n_events), lo, hi)


def serving_pileups(seed: int, n_events: int, lo: int = 50, hi: int = 200) -> np.ndarray:
    """Per-request pileup for the serving workload: uniform integer in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, n_events)


def concat(events):
    """Concatenate events into the batch layout: (offsets[E+1], x, y, z, layer)."""
    off = np.zeros(len(events) + 1, np.int64)
    off[1:] = np.cumsum([e.n_hits for e in events])
    return (off, np.concatenate([e.x for e in events]), np.concatenate([e.y for e in events]),
            np.concatenate([e.z for e in events]), np.concatenate([e.layer for e in events]))
