// Broken-line refit of the fitted tracks (Sec. 2.2.1 and Fig. 2: a fit of each picked
// group of hits determines the track parameters; the broken-line form is V. Blobel,
// NIM A566 (2006) 14).  The track is its offsets from the circle + line fit at the n
// hits, joined by pieces of one common curvature; the direction changes at the hits are
// multiple-scattering kinks weighted by their expected variance.  The library's reading:
//   [B1] reference = the track's circle + line fit; for hit i, s_i = arc length from
//        the closest approach to the hit's radial projection on the reference circle,
//        eps_i = signed distance from that circle (positive to the left of the motion);
//   [B2] transverse unknowns u_1..u_n, dkappa; between hits u'' + kappa0^2 u = dkappa
//        (first-order departure of a circle from the reference circle), so a segment of
//        length h has end slopes a (u_b - c u_a) - a g dkappa and a (c u_b - u_a) +
//        a g dkappa, c = cos(kappa0 h), a = kappa0 / sin(kappa0 h), g = 2 sin^2(kappa0
//        h / 2) / kappa0^2; kink beta_i = slope after - slope before; chi2_T = sum
//        (eps_i - u_i)^2 / (10 um)^2 + sum beta_i^2 / vartheta_i^2;
//   [B3] z is linear in the arc length along the fitted transverse path, s'_i = s_i -
//        kappa0 int_0^{s_i} u (per segment the parabola through its end offsets with
//        second derivative dkappa); unknowns w_i = z offsets from z0 + cot s', kinks of
//        the straight pieces, errors 20 um (barrel z) and |cot| 20 um (disk r);
//   [B4] Highland theta0 = 13.6 MeV / p sqrt(t) (1 + 0.038 ln t), p and the incidence
//        from the reference, t = x/X0 / cos(incidence) (barrel: direction . radial
//        direction; disk: |cos theta|; floored at 1e-3); vartheta^2 = theta0^2 /
//        sin^2 theta, tau^2 = theta0^2 / sin^4 theta;
//   [B5] parameters at the closest approach continue the first segment backwards:
//        kappa0 + dkappa, phi0 + u'(0), d0 - u(0), cot0 + w'_1, z0 + w(0);
//   [B6] a reference with a non-finite value, |kappa0| < 1e-7 /cm or hits not strictly
//        ordered along s (a step <= 1e-6 cm) keeps its circle + line fit;
//   [B7] passes repeat with the previous result as the reference while a pass changes
//        the curvature by more than 1e-3 relative, at most four (one pass is linear in
//        the departures from its reference, and the first moves low-momentum forward
//        tracks by up to 13 % from the circle fit).
//
// One thread per track.  The geometry, the normal equations and their solution run in
// float64: the residuals are micrometres on coordinates of tens of centimetres, and the
// normal equations mix weights of 1e6 (hits) and 1e4..1e8 (kinks).  The kink variances
// only need a few significant digits and are formed in float32, and so is each hit's
// turning angle from the closest approach (relative error ~1e-7: under 0.1 um of arc on
// 30 cm; the hits' distances from the reference circle stay float64).  Divisions are
// few: 1/kappa0 once per track and one per pivot of the factorisation.  GB300 issues few
// float64 operations per cycle, so the segment trigonometry (|kappa0 h| <= 0.5 on
// nearly every track) uses the Taylor series of cos x, sin x / x and (1 - cos x) / x^2
// (truncation below 1e-15) instead of library calls, and distances use sqrt.  The at
// most 7 (transverse) and 6 (longitudinal) unknowns are solved by an LDL^T
// factorisation held in registers: every loop is unrolled over the largest ntuplet, and
// the unknowns of absent hits are padded with unit diagonal entries so they decouple
// and solve to zero.  Each pass is its own launch over the tracks the previous pass
// listed as still moving (a warp-aggregated append), so a warp never waits for the
// slowest of its tracks; the reference of a later pass is the float32 track the previous
// pass wrote (the result depends on its reference only at second order).
#include <cooperative_groups.h>

#include "brokenline.cuh"

namespace ptca {

namespace {

constexpr int kN = kMaxHits;
constexpr double kSigmaT = 10e-4;  // cm
constexpr double kSigmaL = 20e-4;  // cm
constexpr double kCpt = 0.299792458;
constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr double kPassTol = 1e-3;
constexpr int kMaxPasses = 4;
static_assert(kMaxPasses <= kRefitCounters, "one counter per pass");

// cos x, sin x / x and (1 - cos x) / x^2: Taylor series in x^2 for |x| <= 0.5 (the next
// terms are below 1e-15), the library beyond.
__device__ __forceinline__ void trig3(double x, double& c, double& sc, double& vc) {
  if (fabs(x) <= 0.5) {
    const double t = x * x;
    c = 1.0 + t * (-1.0 / 2 + t * (1.0 / 24 + t * (-1.0 / 720 + t * (1.0 / 40320 +
        t * (-1.0 / 3628800 + t * (1.0 / 479001600))))));
    sc = 1.0 + t * (-1.0 / 6 + t * (1.0 / 120 + t * (-1.0 / 5040 + t * (1.0 / 362880 +
         t * (-1.0 / 39916800 + t * (1.0 / 6227020800.0))))));
    vc = 1.0 / 2 + t * (-1.0 / 24 + t * (1.0 / 720 + t * (-1.0 / 40320 + t * (1.0 / 3628800 +
         t * (-1.0 / 479001600 + t * (1.0 / 87178291200.0))))));
  } else {
    double sn;
    sincos(x, &sn, &c);
    sc = sn / x;
    vc = (1.0 - c) / (x * x);
  }
}

// Solves A v = r for symmetric positive definite A (lower triangle read) by LDL^T;
// r is replaced by v.  One float64 division per pivot (its inverse multiplies).
template <int M>
__device__ __forceinline__ void ldl_solve(double (&A)[M][M], double (&r)[M]) {
  double inv[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k] * A[k][k];
    A[j][j] = d;
    inv[j] = 1.0 / d;
#pragma unroll
    for (int i = j + 1; i < M; ++i) {
      double v = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= A[i][k] * A[j][k] * A[k][k];
      A[i][j] = v * inv[j];
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int k = 0; k < i; ++k) r[i] -= A[i][k] * r[k];
  }
#pragma unroll
  for (int i = 0; i < M; ++i) r[i] *= inv[i];
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
#pragma unroll
    for (int k = i + 1; k < M; ++k) r[i] -= A[k][i] * r[k];
  }
}

// One refit pass of track j from its current fit; writes the result and returns true
// when the pass ran, with *more set when the curvature moved by more than kPassTol.
__device__ __forceinline__ bool refit_pass(const Buffers& b, uint64_t j, double bfield,
                                           double x0b, double x0d, bool* more) {
  *more = false;
  const uint32_t t = b.ord[b.sv[j]];
  const int n = b.nt_n[t];
  pt_track tr = b.tracks[j];
  if (n < 3 || n > kN) return false;
  {
    float xf[kN], yf[kN];
    double x[kN], y[kN], z[kN];
    bool barrel[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      xf[i] = yf[i] = 0.0f;
      z[i] = 0.0;
      barrel[i] = true;
      if (i < n) {
        const int32_t g = b.nt_hits[(uint64_t)t * kMaxHits + i];
        xf[i] = b.in_x[g];
        yf[i] = b.in_y[g];
        z[i] = b.in_z[g];
        barrel[i] = b.in_layer[g] < 4;
      }
      x[i] = xf[i];
      y[i] = yf[i];
    }
    // reference of this pass
    double k0 = tr.kappa, phi0 = tr.phi0, d0 = tr.d0, cot0 = tr.cot_theta, z00 = tr.z0;
    double chi2t = 0.0, chi2l = 0.0;
    {
      // [B6]
      if (!isfinite(k0) || !isfinite(phi0) || !isfinite(d0) || !isfinite(cot0) ||
          !isfinite(z00) || fabs(k0) < 1e-7)
        return false;
      // [B1] arc lengths and transverse residuals
      double sp0, cp0;
      sincos(phi0, &sp0, &cp0);
      const double ik0 = 1.0 / k0;  // the one float64 division of the geometry
      const double ccen = d0 - ik0;
      const double cx = ccen * sp0, cy = -ccen * cp0;
      const double ax = sp0 * ik0, ay = -cp0 * ik0;
      const double sgn = k0 > 0.0 ? 1.0 : -1.0, rad = fabs(ik0);
      double s[kN], eps[kN];
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        s[i] = eps[i] = 0.0;
        if (i < n) {
          const double bx = x[i] - cx, by = y[i] - cy;
          // the turning angle from the closest approach in float32 (relative error ~1e-7:
          // under 0.1 um of arc length on 30 cm), the rest of the arc in float64
          s[i] = (double)atan2f((float)(ax * by - ay * bx), (float)(ax * bx + ay * by)) * ik0;
          eps[i] = sgn * (rad - sqrt(bx * bx + by * by));
        }
      }
      double h[kN - 1];
      bool ordered = true;
#pragma unroll
      for (int i = 0; i < kN - 1; ++i) {
        h[i] = 1.0;
        if (i + 1 < n) {
          h[i] = s[i + 1] - s[i];
          ordered = ordered && h[i] > 1e-6;
        }
      }
      if (!ordered) return false;
      // [B4] kink variances at the interior hits (float32)
      const double sth = 1.0 / sqrt(1.0 + cot0 * cot0);
      const float sthf = (float)sth, cthf = (float)(cot0 * sth);
      const float pf = (float)(kCpt * bfield / (100.0 * fabs(k0)) / sth);
      double wt[kN], wl[kN];  // inverse variances
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        wt[i] = wl[i] = 0.0;
        if (i >= 1 && i + 1 < n) {
          float tx;
          if (barrel[i]) {
            float sps, cps;
            sincosf((float)(phi0 + k0 * s[i]), &sps, &cps);
            const float cos_inc = fabsf(sthf * (cps * xf[i] + sps * yf[i])) /
                                  sqrtf(xf[i] * xf[i] + yf[i] * yf[i]);
            tx = (float)x0b / fmaxf(cos_inc, 1e-3f);
          } else {
            tx = (float)x0d / fmaxf(fabsf(cthf), 1e-3f);
          }
          const float th0 = 0.0136f / pf * sqrtf(tx) * (1.0f + 0.038f * logf(tx));
          const float inv = (sthf * sthf) / (th0 * th0);
          wt[i] = inv;
          wl[i] = (double)inv * (double)(sthf * sthf);
        }
      }
      // [B2] segment coefficients c, a and g
      double sc[kN - 1], sa[kN - 1], sg[kN - 1];
#pragma unroll
      for (int i = 0; i < kN - 1; ++i) {
        double snc, vc;
        trig3(k0 * h[i], sc[i], snc, vc);
        sa[i] = 1.0 / (h[i] * snc);
        sg[i] = h[i] * h[i] * vc;
      }
      // transverse normal equations: unknowns u_0..u_5, dkappa (index kN)
      double A[kN + 1][kN + 1];
      double r[kN + 1];
#pragma unroll
      for (int i = 0; i <= kN; ++i) {
        r[i] = 0.0;
#pragma unroll
        for (int k = 0; k <= i; ++k) A[i][k] = 0.0;
      }
      const double wm = 1.0 / (kSigmaT * kSigmaT);
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        A[i][i] = i < n ? wm : 1.0;
        r[i] = i < n ? eps[i] * wm : 0.0;
      }
#pragma unroll
      for (int i = 1; i < kN - 1; ++i) {
        if (i + 1 < n) {
          const double q0 = sa[i - 1], q1 = -(sa[i] * sc[i] + sa[i - 1] * sc[i - 1]);
          const double q2 = sa[i], q3 = -(sa[i] * sg[i] + sa[i - 1] * sg[i - 1]);
          const double w = wt[i];
          A[i - 1][i - 1] += w * q0 * q0;
          A[i][i - 1] += w * q1 * q0;
          A[i + 1][i - 1] += w * q2 * q0;
          A[kN][i - 1] += w * q3 * q0;
          A[i][i] += w * q1 * q1;
          A[i + 1][i] += w * q2 * q1;
          A[kN][i] += w * q3 * q1;
          A[i + 1][i + 1] += w * q2 * q2;
          A[kN][i + 1] += w * q3 * q2;
          A[kN][kN] += w * q3 * q3;
        }
      }
      ldl_solve(A, r);
      double u[kN];
#pragma unroll
      for (int i = 0; i < kN; ++i) u[i] = r[i];
      const double dk = r[kN];
      double c2t = 0.0;
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        if (i < n) c2t += (eps[i] - u[i]) * (eps[i] - u[i]) * wm;
        if (i >= 1 && i + 1 < n) {
          const double beta = sa[i] * (u[i + 1] - sc[i] * u[i]) - sa[i] * sg[i] * dk -
                              (sa[i - 1] * (sc[i - 1] * u[i] - u[i - 1]) +
                               sa[i - 1] * sg[i - 1] * dk);
          c2t += beta * beta * wt[i];
        }
      }
      // [B5] transverse parameters at the closest approach
      const double du1 = sa[0] * (u[1] - sc[0] * u[0]) - sa[0] * sg[0] * dk;
      double cs, snc0, vc0;
      trig3(k0 * s[0], cs, snc0, vc0);
      const double snk = s[0] * snc0;
      const double gs = s[0] * s[0] * vc0;
      const double u0 = u[0] * cs + gs * dk - du1 * snk;
      const double du0 = du1 * cs + k0 * k0 * u[0] * snk - dk * snk;
      // [B3] arc lengths along the fitted transverse path, z residuals
      double sp[kN];
      double acc = s[0] * (u0 + u[0]) * 0.5 - dk * s[0] * s[0] * s[0] * (1.0 / 12.0);
      sp[0] = s[0] - k0 * acc;
#pragma unroll
      for (int i = 1; i < kN; ++i) {
        sp[i] = 0.0;
        if (i < n) {
          const double hh = h[i - 1];
          acc += hh * (u[i - 1] + u[i]) * 0.5 - dk * hh * hh * hh * (1.0 / 12.0);
          sp[i] = s[i] - k0 * acc;
        }
      }
      double hp[kN - 1], ih[kN - 1];
#pragma unroll
      for (int i = 0; i < kN - 1; ++i) {
        hp[i] = i + 1 < n ? sp[i + 1] - sp[i] : 1.0;
        ih[i] = 1.0 / hp[i];
      }
      double B[kN][kN];
      double c[kN];
#pragma unroll
      for (int i = 0; i < kN; ++i) {
#pragma unroll
        for (int k = 0; k <= i; ++k) B[i][k] = 0.0;
      }
      double dl[kN], wz[kN];
      const double wzb = 1.0 / (kSigmaL * kSigmaL);
      const double sld = fmax(fabs(cot0) * kSigmaL, 1e-12);
      const double wzd = 1.0 / (sld * sld);
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        dl[i] = 0.0;
        wz[i] = 0.0;
        if (i < n) {
          wz[i] = barrel[i] ? wzb : wzd;
          dl[i] = z[i] - (z00 + cot0 * sp[i]);
        }
        B[i][i] = i < n ? wz[i] : 1.0;
        c[i] = dl[i] * wz[i];
      }
#pragma unroll
      for (int i = 1; i < kN - 1; ++i) {
        if (i + 1 < n) {
          const double q0 = ih[i - 1], q2 = ih[i], q1 = -(q0 + q2);
          const double w = wl[i];
          B[i - 1][i - 1] += w * q0 * q0;
          B[i][i - 1] += w * q1 * q0;
          B[i + 1][i - 1] += w * q2 * q0;
          B[i][i] += w * q1 * q1;
          B[i + 1][i] += w * q2 * q1;
          B[i + 1][i + 1] += w * q2 * q2;
        }
      }
      ldl_solve(B, c);
      double c2l = 0.0;
#pragma unroll
      for (int i = 0; i < kN; ++i) {
        if (i < n) c2l += (dl[i] - c[i]) * (dl[i] - c[i]) * wz[i];
        if (i >= 1 && i + 1 < n) {
          const double g = (c[i + 1] - c[i]) * ih[i] - (c[i] - c[i - 1]) * ih[i - 1];
          c2l += g * g * wl[i];
        }
      }
      const double dw1 = (c[1] - c[0]) * ih[0];
      const double kappa = k0 + dk;
      const double change = fabs(dk) / fabs(k0);
      k0 = kappa;
      phi0 = remainder(phi0 + du0, kTwoPi);
      d0 = d0 - u0;
      z00 = z00 + c[0] - sp[0] * dw1;
      cot0 = cot0 + dw1;
      chi2t = c2t;
      chi2l = c2l;
      *more = change > kPassTol;
    }
    tr.kappa = (float)k0;
    tr.phi0 = (float)phi0;
    tr.d0 = (float)d0;
    tr.cot_theta = (float)cot0;
    tr.z0 = (float)z00;
    tr.pt = (float)(kCpt * bfield / (100.0 * fabs(k0)));
    tr.chi2_circle = (float)chi2t;
    tr.chi2_line = (float)chi2l;
    tr.charge = k0 > 0.0 ? -1 : (k0 < 0.0 ? 1 : 0);
    b.tracks[j] = tr;
  }
  return true;
}

// One pass over every cleaned track (in_list null) or over the in_n[0] tracks of
// in_list; tracks that keep moving are appended to out_list (when given).
__global__ void __launch_bounds__(128) k_refit_bl(Buffers b, double bfield, double x0b,
                                                   double x0d, const uint32_t* in_list,
                                                   const unsigned long long* in_n,
                                                   uint32_t* out_list,
                                                   unsigned long long* out_n, uint64_t cap) {
  namespace cg = cooperative_groups;
  const uint64_t N = min(in_list ? *in_n : b.cnt[CNT_SV], (unsigned long long)cap);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const uint64_t j = in_list ? in_list[i] : i;
    bool more;
    refit_pass(b, j, bfield, x0b, x0d, &more);
    if (more && out_list) {
      cg::coalesced_group g = cg::coalesced_threads();
      unsigned long long base = 0;
      if (g.thread_rank() == 0) base = atomicAdd(out_n, (unsigned long long)g.size());
      base = g.shfl(base, 0);
      out_list[base + g.thread_rank()] = (uint32_t)j;
    }
  }
}

}  // namespace

cudaError_t launch_refit_broken_line(const Buffers& b, const Params& p, float x0_barrel,
                                     float x0_disk, uint32_t* list, unsigned long long* counters,
                                     const Launch& l, cudaStream_t s) {
  const uint64_t cap = (uint64_t)p.max_ntuplets;
  uint32_t* lists[2] = {list, list + cap};
  const cudaError_t e = cudaMemsetAsync(counters, 0, kMaxPasses * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    const uint32_t* in = pass == 0 ? nullptr : lists[(pass - 1) & 1];
    const unsigned long long* in_n = pass == 0 ? nullptr : &counters[pass - 1];
    uint32_t* out = pass + 1 < kMaxPasses ? lists[pass & 1] : nullptr;
    unsigned long long* out_n = pass + 1 < kMaxPasses ? &counters[pass] : nullptr;
    PT_TRACE(l, s, "k_refit_bl",
             k_refit_bl<<<l.sms * 8, 128, 0, s>>>(b, (double)p.bfield, (double)x0_barrel,
                                                   (double)x0_disk, in, in_n, out, out_n, cap));
  }
  return cudaGetLastError();
}

}  // namespace ptca
