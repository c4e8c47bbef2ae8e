"""Seeded synthetic pixel events: charged helices in a solenoid, plus uniform noise.

This module is the input recipe shared by the tests, the benchmark and the gate
training script.  It contains no reconstruction arithmetic: it draws particles, intersects
their helices with the detector surfaces and smears the crossings.

Units: cm, GeV, tesla.  Magnetic field along +z.

Multiple scattering (off unless a configuration gives material): every surface a
particle crosses holds x0 radiation lengths at normal incidence (x0_barrel, x0_disk);
at each crossing the direction is turned by two independent Gaussian angles of RMS
theta0 = 13.6 MeV / p sqrt(t) (1 + 0.038 ln t), t = x0 / cos(incidence) (the Highland
formula, beta = 1), in the two planes through the direction, and the helix continues
from the crossing with the same momentum.

Detector (layer codes are part of the library's input contract):
  0..3  barrel cylinders, r = 2.9 / 6.8 / 10.9 / 16.0 cm, |z| < 27 cm
  4..6  disks at z = +29.1 / +39.6 / +51.6 cm, 4.5 <= r <= 16 cm
  7..9  disks at z = -29.1 / -39.6 / -51.6 cm, same radial extent

Overlapping sensors (off unless a configuration gives `overlap`): a crossing falls in the
overlap of two neighbouring sensors of its layer with probability `overlap`, and the
particle then also crosses the second sensor, which sits OVERLAP_DR further out (barrel)
or OVERLAP_DZ further from z = 0 (disks), leaving a second hit with the same layer code.

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

OVERLAP_DR = 0.5    # cm, radial offset of a barrel layer's overlapping sensors
OVERLAP_DZ = 0.5    # cm, z offset of a disk's overlapping sensors

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
    x0_barrel: float = 0.0  # radiation lengths per barrel layer (0: no scattering)
    x0_disk: float = 0.0    # radiation lengths per disk
    hit_eff: float = 1.0    # probability that a crossing gives a hit (1: every crossing)
    overlap: float = 0.0    # probability that a crossing also crosses an overlapping sensor


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


def _overlap_crossings(p: dict, pid, lay):
    """Noiseless crossings of the overlapping sensors behind the given crossings
    (pid, layer): barrel radius + OVERLAP_DR, disk |z| + OVERLAP_DZ.  Returns
    (pid, layer, x, y, z) of those that lie inside the sensor's acceptance."""
    R, z0, q = p["R"][pid], p["z0"][pid], p["q"][pid]
    sh, phi0 = np.sinh(p["eta"][pid]), p["phi0"][pid]
    barrel = lay < 4
    rl = np.asarray(BARREL_R + (0.0,) * 6)[lay] + OVERLAP_DR
    ok_b = barrel & (rl < 2.0 * R)
    alpha_b = 2.0 * np.arcsin(np.where(ok_b, rl / (2.0 * R), 0.0))
    zb = z0 + R * alpha_b * sh
    ok_b &= np.abs(zb) < BARREL_ZMAX
    side = np.where(lay < 7, 1.0, -1.0)
    zd = side * (np.asarray((0.0,) * 4 + DISK_Z + DISK_Z)[lay] + OVERLAP_DZ)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_d = (zd - z0) / sh
    alpha_d = np.where(np.isfinite(s_d), s_d / R, -1.0)
    ok_d = ~barrel & np.isfinite(s_d) & (s_d > 0) & (alpha_d < np.pi)
    rd = 2.0 * R * np.sin(np.where(ok_d, alpha_d, 0.0) / 2.0)
    ok_d &= (rd >= DISK_RMIN) & (rd <= DISK_RMAX)
    alpha = np.where(barrel, alpha_b, alpha_d)
    r = np.where(barrel, rl, rd)
    z = np.where(barrel, zb, zd)
    phi = phi0 - q * alpha / 2.0
    keep = ok_b | ok_d
    return (pid[keep], lay[keep], r[keep] * np.cos(phi[keep]), r[keep] * np.sin(phi[keep]),
            z[keep])


def highland(p, t):
    """RMS plane scattering angle (rad) of a momentum-p (GeV) particle with beta = 1
    through t radiation lengths."""
    return 0.0136 / p * np.sqrt(t) * (1.0 + 0.038 * np.log(t))


def _crossings_ms(rng, p: dict, barrel_only: bool, x0_barrel: float, x0_disk: float):
    """Crossings with multiple scattering, surface by surface along each helix.  Returns
    (pid, layer, x, y, z, step) float64 arrays; step orders each particle's crossings.

    State per particle: position, transverse direction psi (motion turns by -q s / R),
    dz/ds = cot, radius R.  The next crossing is the smallest positive arc length to an
    unused surface within its acceptance, while the total turning stays below pi (the
    outgoing half turn, as without material)."""
    n = p["pt"].shape[0]
    pmag = p["pt"] * np.cosh(p["eta"])
    px, py, pz = np.zeros(n), np.zeros(n), p["z0"].copy()
    psi = p["phi0"].copy()
    cot = np.sinh(p["eta"])
    R = p["R"].copy()
    q = p["q"]
    turned = np.zeros(n)
    alive = np.ones(n, bool)
    surfaces = [("barrel", r, L) for L, r in enumerate(BARREL_R)]
    if not barrel_only:
        surfaces += [("disk", zd, 4 + k) for k, zd in enumerate(DISK_Z)]
        surfaces += [("disk", -zd, 7 + k) for k, zd in enumerate(DISK_Z)]
    used = np.zeros((n, len(surfaces)), bool)
    out = []
    for step in range(len(surfaces)):
        # centre of the transverse circle and arc length to each surface
        cx = px + q * R * np.sin(psi)
        cy = py - q * R * np.cos(psi)
        a0 = np.arctan2(py - cy, px - cx)
        cand = np.full((n, len(surfaces)), np.inf)
        for j, (kind, v, L) in enumerate(surfaces):
            if kind == "barrel":
                cc = np.hypot(cx, cy)
                with np.errstate(divide="ignore", invalid="ignore"):
                    K = (v * v - cc * cc - R * R) / (2.0 * R * cc)
                ok = np.abs(K) <= 1.0
                gam = np.arctan2(cy, cx)
                acs = np.arccos(np.clip(K, -1.0, 1.0))
                best = np.full(n, np.inf)
                for sgn in (1.0, -1.0):
                    a = gam + sgn * acs
                    turn = np.remainder(q * (a0 - a), 2.0 * np.pi)
                    turn = np.where(turn < 1e-12, turn + 2.0 * np.pi, turn)
                    best = np.minimum(best, np.where(ok, turn, np.inf))
                s = R * best
                zc = pz + cot * s
                inside = np.abs(zc) < BARREL_ZMAX
            else:
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = (v - pz) / cot
                ok = np.isfinite(s) & (s > 1e-9)
                aa = a0 - q * np.where(ok, s, 0.0) / R
                s = np.where(ok, s, np.inf)
                xc = cx + R * np.cos(aa)
                yc = cy + R * np.sin(aa)
                rc = np.hypot(xc, yc)
                inside = (rc >= DISK_RMIN) & (rc <= DISK_RMAX)
            good = np.isfinite(s) & inside & ~used[:, j] & (turned + s / R < np.pi)
            cand[:, j] = np.where(good, s, np.inf)
        j = np.argmin(cand, axis=1)
        s = cand[np.arange(n), j]
        hit = alive & np.isfinite(s)
        alive = hit
        g1 = rng.normal(0.0, 1.0, n)
        g2 = rng.normal(0.0, 1.0, n)
        if not hit.any():
            break
        s = np.where(hit, s, 0.0)
        aa = a0 - q * s / R
        nx = cx + R * np.cos(aa)
        ny = cy + R * np.sin(aa)
        nz = pz + cot * s
        npsi = psi - q * s / R
        lay = np.asarray([surfaces[k][2] for k in j])
        idx = np.flatnonzero(hit)
        out.append((idx, lay[idx], nx[idx], ny[idx], nz[idx], np.full(idx.size, step)))
        used[idx, j[idx]] = True
        # scattering at the crossing
        sth = 1.0 / np.sqrt(1.0 + cot * cot)
        cth = cot * sth
        d = np.stack([sth * np.cos(npsi), sth * np.sin(npsi), cth])
        barrel = lay < 4
        rr = np.hypot(nx, ny)
        cos_inc = np.where(barrel, np.abs(d[0] * nx + d[1] * ny) / np.where(rr > 0, rr, 1.0),
                           np.abs(cth))
        x0 = np.where(barrel, x0_barrel, x0_disk)
        t = x0 / np.maximum(cos_inc, 1e-6)
        th0 = np.where(x0 > 0, highland(pmag, np.where(x0 > 0, t, 1.0)), 0.0)
        e1 = np.stack([-np.sin(npsi), np.cos(npsi), np.zeros(n)])
        e2 = np.stack([cth * np.cos(npsi), cth * np.sin(npsi), -sth])
        dn = d + (g1 * th0) * e1 + (g2 * th0) * e2
        dn /= np.linalg.norm(dn, axis=0)
        st = np.hypot(dn[0], dn[1])
        upd = hit
        px = np.where(upd, nx, px)
        py = np.where(upd, ny, py)
        pz = np.where(upd, nz, pz)
        psi = np.where(upd, np.arctan2(dn[1], dn[0]), psi)
        cot = np.where(upd, dn[2] / st, cot)
        turned = np.where(upd, turned + s / R, turned)
        R = np.where(upd, pmag * st / (C_LIGHT * BFIELD_T) * 100.0, R)
    if not out:
        e = np.zeros(0)
        return e.astype(np.int32), e.astype(np.uint8), e, e, e, e.astype(np.int64)
    pid = np.concatenate([o[0] for o in out]).astype(np.int32)
    lay = np.concatenate([o[1] for o in out]).astype(np.uint8)
    x = np.concatenate([o[2] for o in out])
    y = np.concatenate([o[3] for o in out])
    z = np.concatenate([o[4] for o in out])
    st = np.concatenate([o[5] for o in out]).astype(np.int64)
    return pid, lay, x, y, z, st


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
    if cfg.x0_barrel > 0.0 or cfg.x0_disk > 0.0:
        pid, lay, xt, yt, zt, _ = _crossings_ms(rng, p, cfg.barrel_only, cfg.x0_barrel,
                                                cfg.x0_disk)
    else:
        pid, lay, xt, yt, zt = _crossings(p, cfg.barrel_only)
    if cfg.overlap > 0.0:
        if cfg.x0_barrel > 0.0 or cfg.x0_disk > 0.0:
            raise ValueError("overlapping sensors are modelled without material only")
        sel = rng.random(pid.shape[0]) < cfg.overlap
        o = _overlap_crossings(p, pid[sel], lay[sel])
        pid, lay, xt, yt, zt = (np.concatenate([a, b]) for a, b in zip((pid, lay, xt, yt, zt), o))
    if cfg.hit_eff < 1.0:  # inefficient sensors: each crossing kept independently
        keep = rng.random(pid.shape[0]) < cfg.hit_eff
        pid, lay, xt, yt, zt = pid[keep], lay[keep], xt[keep], yt[keep], zt[keep]
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
