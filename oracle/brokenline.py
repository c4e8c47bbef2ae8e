"""CPU oracle of the broken-line refit (float64).

TEST INFRASTRUCTURE ONLY: the tests are the only callers; the product never loads it.
It shares no code with the CUDA path.

Sec. 2.2.1 and Fig. 2: a fit of each picked group of hits determines the track
parameters; the paper prints no fit equations.  This refit takes the broken-line form
(V. Blobel, NIM A566 (2006) 14): the track is described by its offsets from a
reference trajectory at the n measurement planes, joined by pieces of one common
curvature whose direction changes at the planes are multiple-scattering kinks, each
weighted by its expected variance; the offsets, the curvature correction and the
kinks follow from one linear least-squares problem.  The library's reading:

  [B1] Reference: the circle + line fit (kappa0, phi0, d0, cot0, z00).  Circle centre
       C = (d0 - 1/kappa0) n and closest approach d0 n, n = (sin phi0, -cos phi0).  For
       hit i (inner to outer): s_i = arc length from the closest approach along the
       reference circle to the hit's radial projection, eps_i = signed distance of the
       hit from the circle (positive to the left of the motion), delta_i = z_i - (z00 +
       cot0 s_i); h_i = s_{i+1} - s_i.
  [B2] Transverse plane: unknowns u_1..u_n (offsets, positive to the left) and dkappa.
       Between planes a circle of curvature kappa0 + dkappa departs from the reference
       circle, to first order, by u(s) with u'' + kappa0^2 u = dkappa (a parabola of
       second derivative dkappa as kappa0 -> 0).  On a segment of length h with end
       offsets u_a, u_b the end slopes are
         u'(start) = a (u_b - c u_a) - a g dkappa,  u'(end) = a (c u_b - u_a) + a g dkappa,
       c = cos(kappa0 h), a = kappa0 / sin(kappa0 h), g = 2 sin^2(kappa0 h / 2) / kappa0^2
       (-> 1/h and h^2/2).  The kink at interior plane i is beta_i = u'(s_i+) - u'(s_i-),
       and chi2_T = sum (eps_i - u_i)^2 / sigma_T^2 + sum beta_i^2 / vartheta_i^2,
       sigma_T = 10 um.
  [B3] Longitudinal: z is linear in the arc length along the fitted transverse path,
       s'_i = s_i - kappa0 int_0^{s_i} u ds (a left offset shortens the path when the
       centre is on the left), u integrated per segment as the parabola through its end
       offsets with second derivative dkappa (from the closest approach to the first
       plane through u(0) of [B5]).  Unknowns w_1..w_n (z offsets from z00 + cot0 s'),
       h'_i = s'_{i+1} - s'_i, kinks gamma_i = (w_{i+1} - w_i)/h'_i - (w_i - w_{i-1})/h'_{i-1},
       chi2_L = sum (delta_i - w_i)^2 / sigma_L,i^2 + sum gamma_i^2 / tau_i^2,
       delta_i = z_i - (z00 + cot0 s'_i), sigma_L = 20 um on a barrel hit (its z) and
       |cot0| x 20 um on a disk hit (its r error moved along the line).
  [B4] Kink variances from the Highland formula, theta0 = 13.6 MeV / p sqrt(t) (1 +
       0.038 ln t), with p = pT / sin(theta) of the reference (pT = 0.299792458 B /
       (100 |kappa0|) GeV) and t = x/X0 / cos(incidence): on a barrel layer the cosine
       between the reference direction at s_i and the radial direction of the hit, on
       a disk |cos theta| (floored at 1e-3).  A scattering angle theta0 turns the
       transverse direction by theta0 / sin(theta) and dz/ds by theta0 / sin^2(theta):
       vartheta_i^2 = theta0^2 / sin^2(theta), tau_i^2 = theta0^2 / sin^4(theta).
  [B5] Parameters at the closest approach, continuing the first segment backwards (no
       material inside the first plane), with u'_1 = u'(s_1+):
         u(0) = u_1 cos(kappa0 s_1) + g(s_1) dkappa - u'_1 sin(kappa0 s_1) / kappa0,
         u'(0) = u'_1 cos(kappa0 s_1) + (kappa0 u_1 - dkappa / kappa0) sin(kappa0 s_1);
       kappa = kappa0 + dkappa, phi0 + u'(0), d0 - u(0); w'_1 = (w_2 - w_1)/h'_1,
       cot = cot0 + w'_1, z0 = z00 + w_1 - s'_1 w'_1.  chi2_circle = chi2_T and
       chi2_line = chi2_L at the minimum; charge = -sign(kappa).
  [B6] A track with fewer than 3 hits, a reference with a non-finite value, |kappa0| <
       1e-7 cm^-1 or some h_i <= 1e-6 cm keeps its reference fit.
  [B7] The refit repeats with its own result as the reference while a pass changes the
       curvature by more than 1e-3 relative, at most four passes: one pass is linear
       in the departures from the reference, and on low-momentum forward tracks the
       first pass moves the curvature by up to 13 % from the circle fit; each further
       pass shrinks the change about tenfold or better, so the result lies within a
       few 1e-5 of the converged one.
"""

from __future__ import annotations

import math

import numpy as np

SIGMA_T = 10e-4  # cm
SIGMA_L = 20e-4  # cm
C_PT = 0.299792458


def highland(p: float, t: float) -> float:
    """[B4] RMS plane scattering angle (rad) at momentum p (GeV) through t X0."""
    return 0.0136 / p * math.sqrt(t) * (1.0 + 0.038 * math.log(t))


def reference_geometry(x, y, z, ref):
    """[B1] Arc lengths s, transverse residuals eps and z residuals delta of the hits
    with respect to the reference (kappa0, phi0, d0, cot0, z00)."""
    k0, phi0, d0, cot0, z00 = (float(v) for v in ref[:5])
    nx, ny = math.sin(phi0), -math.cos(phi0)
    cx, cy = (d0 - 1.0 / k0) * nx, (d0 - 1.0 / k0) * ny
    ax, ay = nx / k0, ny / k0  # closest approach - centre
    s, eps, delta = [], [], []
    for xi, yi, zi in zip(x, y, z):
        bx, by = float(xi) - cx, float(yi) - cy
        si = math.atan2(ax * by - ay * bx, ax * bx + ay * by) / k0
        s.append(si)
        eps.append(math.copysign(1.0, k0) * (1.0 / abs(k0) - math.hypot(bx, by)))
        delta.append(float(zi) - (z00 + cot0 * si))
    return np.asarray(s), np.asarray(eps), np.asarray(delta)


def kink_variances(x, y, layer, s, ref, x0_barrel, x0_disk, bfield):
    """[B4] (vartheta_i^2, tau_i^2) at every hit (used at the interior ones)."""
    k0, phi0, _, cot0, _ = (float(v) for v in ref[:5])
    sth = 1.0 / math.sqrt(1.0 + cot0 * cot0)
    cth = cot0 * sth
    p = C_PT * bfield / (100.0 * abs(k0)) / sth
    vt, vl = [], []
    for xi, yi, li, si in zip(x, y, layer, s):
        if int(li) < 4:
            psi = phi0 + k0 * si
            r = math.hypot(float(xi), float(yi))
            cos_inc = abs(sth * (math.cos(psi) * float(xi) + math.sin(psi) * float(yi))) / r
            t = x0_barrel / max(cos_inc, 1e-3)
        else:
            t = x0_disk / max(abs(cth), 1e-3)
        th0 = highland(p, t)
        vt.append(th0 * th0 / (sth * sth))
        vl.append(th0 * th0 / (sth ** 4))
    return np.asarray(vt), np.asarray(vl)


def _sinc(x: float) -> float:
    return math.sin(x) / x if abs(x) > 1e-4 else 1.0 - x * x / 6.0


def segment(k0: float, h: float):
    """[B2] (c, a, g) of a segment of length h on the reference of curvature k0."""
    c = math.cos(k0 * h)
    a = 1.0 / (h * _sinc(k0 * h))
    g = 0.5 * h * h * _sinc(0.5 * k0 * h) ** 2
    return c, a, g


def _solve(A, b):
    """Least-squares solution, chi2 and covariance (A^T A)^-1 of the weighted rows."""
    v = np.linalg.lstsq(A, b, rcond=None)[0]
    r = A @ v - b
    return v, float(r @ r), np.linalg.inv(A.T @ A)


def refit(x, y, z, layer, ref, x0_barrel: float, x0_disk: float, bfield: float = 3.8,
          sigma_t: float = SIGMA_T, sigma_l: float = SIGMA_L, full: bool = False):
    """Broken-line refit of one track (hits inner to outer; ref = the circle + line fit's
    first five values, or its nine).  Returns the nine fit values (kappa, phi0, d0,
    cot_theta, z0, pt, chi2_circle, chi2_line, charge); with full=True also a dict of
    the solution (u, dkappa, w, beta, gamma, s, covariances)."""
    n = len(x)
    ref = np.asarray(ref, np.float64)
    keep = np.concatenate([ref[:5], [C_PT * bfield / (100.0 * abs(ref[0])) if ref[0] else math.inf],
                           ref[6:8] if ref.size >= 8 else [0.0, 0.0],
                           [-math.copysign(1.0, ref[0]) if ref[0] else 0.0]])
    if n < 3 or not np.all(np.isfinite(ref[:5])) or abs(ref[0]) < 1e-7:  # [B6]
        return (keep, None) if full else keep
    s, eps, _ = reference_geometry(x, y, z, ref)
    h = np.diff(s)
    if np.any(h <= 1e-6):  # [B6]
        return (keep, None) if full else keep
    vt, vl = kink_variances(x, y, layer, s, ref, x0_barrel, x0_disk, bfield)
    # [B2] transverse rows: n measurements, n - 2 kinks; unknowns u_1..u_n, dkappa
    k0 = float(ref[0])
    seg = [segment(k0, hh) for hh in h]
    A = np.zeros((2 * n - 2, n + 1))
    b = np.zeros(2 * n - 2)
    for i in range(n):
        A[i, i] = 1.0 / sigma_t
        b[i] = eps[i] / sigma_t
    for i in range(1, n - 1):
        w = 1.0 / math.sqrt(vt[i])
        (cp, ap, gp), (cn, an, gn) = seg[i - 1], seg[i]
        row = n + i - 1
        A[row, i - 1] = w * ap
        A[row, i] = -w * (an * cn + ap * cp)
        A[row, i + 1] = w * an
        A[row, n] = -w * (an * gn + ap * gp)
    v, chi2_t, cov_t = _solve(A, b)
    u, dk = v[:n], v[n]
    # [B5] transverse parameters at the closest approach
    c1, a1, g1 = seg[0]
    du1 = a1 * (u[1] - c1 * u[0]) - a1 * g1 * dk
    cs, sn_k = math.cos(k0 * s[0]), s[0] * _sinc(k0 * s[0])
    gs = 0.5 * s[0] ** 2 * _sinc(0.5 * k0 * s[0]) ** 2
    u0 = u[0] * cs + gs * dk - du1 * sn_k
    du0 = du1 * cs + (k0 * u[0] * sn_k * k0 - dk * sn_k)
    # [B3] arc lengths along the fitted transverse path
    sp = np.empty(n)
    acc = s[0] * (u0 + u[0]) / 2.0 - dk * s[0] ** 3 / 12.0
    sp[0] = s[0] - k0 * acc
    for i in range(1, n):
        acc += h[i - 1] * (u[i - 1] + u[i]) / 2.0 - dk * h[i - 1] ** 3 / 12.0
        sp[i] = s[i] - k0 * acc
    hp = np.diff(sp)
    delta = np.asarray(z, np.float64) - (ref[4] + ref[3] * sp)
    sl = np.where(np.asarray(layer) < 4, sigma_l, abs(ref[3]) * sigma_l)
    sl = np.maximum(sl, 1e-12)
    B = np.zeros((2 * n - 2, n))
    c = np.zeros(2 * n - 2)
    for i in range(n):
        B[i, i] = 1.0 / sl[i]
        c[i] = delta[i] / sl[i]
    for i in range(1, n - 1):
        w = 1.0 / math.sqrt(vl[i])
        row = n + i - 1
        B[row, i - 1] = w / hp[i - 1]
        B[row, i] = -w * (1.0 / hp[i - 1] + 1.0 / hp[i])
        B[row, i + 1] = w / hp[i]
    wv, chi2_l, cov_l = _solve(B, c)
    kappa = ref[0] + dk
    phi = math.remainder(ref[1] + du0, 2.0 * math.pi)
    dw1 = (wv[1] - wv[0]) / hp[0]
    out = np.array([kappa, phi, ref[2] - u0, ref[3] + dw1, ref[4] + wv[0] - sp[0] * dw1,
                    C_PT * bfield / (100.0 * abs(kappa)), chi2_t, chi2_l,
                    -math.copysign(1.0, kappa)])
    if not full:
        return out
    beta = np.array([(seg[i][1] * (u[i + 1] - seg[i][0] * u[i]) - seg[i][1] * seg[i][2] * dk)
                     - (seg[i - 1][1] * (seg[i - 1][0] * u[i] - u[i - 1])
                        + seg[i - 1][1] * seg[i - 1][2] * dk) for i in range(1, n - 1)])
    gamma = np.array([(wv[i + 1] - wv[i]) / hp[i] - (wv[i] - wv[i - 1]) / hp[i - 1]
                      for i in range(1, n - 1)])
    gc = np.zeros(n)  # d cot / d w
    gc[0], gc[1] = -1.0 / hp[0], 1.0 / hp[0]
    return out, dict(u=u, dkappa=dk, w=wv, beta=beta, gamma=gamma, s=s, s_path=sp, eps=eps,
                     delta=delta, var_kappa=float(cov_t[n, n]), var_cot=float(gc @ cov_l @ gc),
                     var_t=vt, var_l=vl)


PASS_TOL = 1e-3
MAX_PASSES = 4


def refit_iterated(x, y, z, layer, ref, x0_barrel: float, x0_disk: float,
                   bfield: float = 3.8) -> np.ndarray:
    """[B7] Refit passes, each on the previous result, until the curvature changes by at
    most PASS_TOL relative (MAX_PASSES at most).  Returns the nine fit values."""
    cur = np.asarray(ref, np.float64)
    for _ in range(MAX_PASSES):
        nxt = refit(x, y, z, layer, cur, x0_barrel, x0_disk, bfield)
        change = abs(nxt[0] - cur[0]) / abs(cur[0]) if cur[0] != 0 else 0.0
        cur = nxt
        if not change > PASS_TOL:
            break
    return cur


def refit_tracks(x, y, z, layer, hits, nhits, fits, x0_barrel, x0_disk, bfield=3.8):
    """[B7] Iterated refit of many tracks: hits [T, 6] indices into the hit arrays (inner
    to outer), nhits [T], fits [T, >= 5] their circle + line fits.  Returns [T, 9]."""
    out = np.empty((len(nhits), 9))
    for t, (hr, nh) in enumerate(zip(hits, nhits)):
        idx = np.asarray(hr[:nh], np.int64)
        out[t] = refit_iterated(x[idx], y[idx], z[idx], layer[idx], fits[t], x0_barrel,
                                x0_disk, bfield)
    return out
