// Stage A7: per-candidate helix fit (Sec. 2.2.1, Fig. 2: each picked group of hits is
// fitted, which yields its track parameters).  Circle in the transverse plane by the closed-form fit of
// V. Karimaki (NIM A305 (1991) 187) with equal weights, then z = z0 + cot(theta) s by
// least squares in the transverse arc length s from the point of closest approach.
//
// Eight lanes per candidate (one hit per lane, <= 6 used), sums by xor shuffles within
// the 8-lane group.  The closed form minimises sum (k r^2 - x sin(phi) + y cos(phi)
// + delta)^2 over (k, phi, delta) with r^2 measured from the beam spot; its solution
// only involves covariances, which are rotation covariant.  The kernel therefore
// evaluates it in float32 in the frame centred on the hits' centroid and rotated onto
// their principal axis: there the perpendicular coordinate v is of the order of the
// sagitta, and the curvature term cov(v, r^2) is formed from small numbers instead of
// as the difference of two large ones.  The algebraic residual of hit i in that frame
// is e_i = k (r_i^2 - <r^2>) - u_i sin(phi') + v_i cos(phi'), from which the distance
// to the circle follows without cancellation.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kSigmaRphi = 10e-4f;  // cm
constexpr float kSigmaZ = 20e-4f;     // cm

// a - b = s + e exactly (s the rounded difference): Knuth's two-sum on (a, -b).
__device__ __forceinline__ float two_diff(float a, float b, float& e) {
  const float s = __fsub_rn(a, b);
  const float bb = __fsub_rn(a, s);
  e = __fadd_rn(__fsub_rn(a, __fadd_rn(s, bb)), __fsub_rn(bb, b));
  return s;
}

// Signed curvature (> 0 counter-clockwise) of the circle through three hits, from the
// cross product of the chords leaving the middle hit, evaluated with float32 operations
// that lose almost nothing to cancellation: the coordinate differences are split into
// rounded value and exact remainder, the 2 x 2 determinant uses the fused multiply-add
// form that recovers the rounding error of one product, and the remainders enter to
// first order.  For a short, nearly straight triplet (a few cm of lever arm, a sagitta
// of tens of micrometres) the plain float32 evaluation loses about 1e-4 relative.
__device__ __forceinline__ float triplet_curvature(float x0, float y0, float x1, float y1,
                                                  float x2, float y2) {
  float axe, aye, bxe, bye;
  const float ax = two_diff(x0, x1, axe), ay = two_diff(y0, y1, aye);
  const float bx = two_diff(x2, x1, bxe), by = two_diff(y2, y1, bye);
  const float w = __fmul_rn(ay, bx);
  const float we = __fmaf_rn(ay, bx, -w);          // ay * bx = w + we exactly
  float cr = __fsub_rn(__fmaf_rn(ax, by, -w), we);  // ax * by - ay * bx
  cr = __fadd_rn(cr, __fsub_rn(__fadd_rn(__fmul_rn(ax, bye), __fmul_rn(axe, by)),
                               __fadd_rn(__fmul_rn(ay, bxe), __fmul_rn(aye, bx))));
  const float cx = __fsub_rn(x2, x0), cy = __fsub_rn(y2, y0);
  const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by);
  const float lc = sqrtf(cx * cx + cy * cy);
  // a = p0 - p1, b = p2 - p1: the hits turn counter-clockwise when a x b < 0
  return -2.0f * cr / (la * lb * lc);
}

__device__ __forceinline__ float gsum(float v) {
  v += __shfl_xor_sync(kFull, v, 4, 8);
  v += __shfl_xor_sync(kFull, v, 2, 8);
  v += __shfl_xor_sync(kFull, v, 1, 8);
  return v;
}

__global__ void __launch_bounds__(256) k_fit(Buffers b, float bfield) {
  const uint64_t S = b.cnt[CNT_SV];
  const int lane = lane_id();
  const int sub = lane & 7;
  const int gbase = lane & ~7;
  const uint64_t ngroups = (uint64_t)gridDim.x * blockDim.x / 8;
  const uint64_t g0 = ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / 8;
  for (uint64_t jw = g0; jw < S; jw += ngroups) {
    const uint64_t j = jw + (lane >> 3);
    const bool active = j < S;
    int n = 3;
    float x = 0.0f, y = 0.0f, z = 0.0f;
    uint32_t t = 0;
    if (active) {
      t = b.ord[b.sv[j]];
      n = b.nt_n[t];
      if (!PT_CHECK(b.cnt, n >= 3 && n <= kMaxHits, DBG_FIT_HITS)) n = 3;
      if (sub < n) {
        const int32_t g = b.nt_hits[(uint64_t)t * kMaxHits + sub];
        x = b.in_x[g];
        y = b.in_y[g];
        z = b.in_z[g];
      }
    }
    const bool valid = sub < n;
    const float inv_n = 1.0f / (float)n;
    // centroid and principal axis
    const float mx = gsum(x) * inv_n, my = gsum(y) * inv_n;
    const float dx = valid ? x - mx : 0.0f, dy = valid ? y - my : 0.0f;
    const float cxx = gsum(dx * dx) * inv_n, cxy = gsum(dx * dy) * inv_n;
    const float cyy = gsum(dy * dy) * inv_n;
    const float al = 0.5f * atan2f(2.0f * cxy, cxx - cyy);
    float sa, ca;
    sincosf(al, &sa, &ca);
    const float du = dx * ca + dy * sa, dv = -dx * sa + dy * ca;
    const float Mt = mx * ca + my * sa, Mn = -mx * sa + my * ca;
    const float w = du * du + dv * dv;
    const float mw = gsum(w) * inv_n;
    const float dr = valid ? 2.0f * Mt * du + 2.0f * Mn * dv + (w - mw) : 0.0f;
    const float mr = Mt * Mt + Mn * Mn + mw;
    const float cuu = gsum(du * du) * inv_n, cuv = gsum(du * dv) * inv_n;
    const float cvv = gsum(dv * dv) * inv_n;
    const float cur = gsum(du * dr) * inv_n, cvr = gsum(dv * dr) * inv_n;
    const float crr = gsum(dr * dr) * inv_n;
    const float q1 = crr * cuv - cur * cvr;
    const float q2 = crr * (cuu - cvv) - cur * cur + cvr * cvr;
    float ph = 0.5f * atan2f(2.0f * q1, q2);
    float s, c;
    sincosf(ph, &s, &c);
    // travel direction: from the first towards the last hit
    const float du0 = __shfl_sync(kFull, du, gbase), dv0 = __shfl_sync(kFull, dv, gbase);
    const float dun = __shfl_sync(kFull, du, gbase + n - 1);
    const float dvn = __shfl_sync(kFull, dv, gbase + n - 1);
    if (c * (dun - du0) + s * (dvn - dv0) < 0.0f) {
      ph = ph > 0.0f ? ph - kPi : ph + kPi;
      s = -s;
      c = -c;
    }
    const float k = (s * cur - c * cvr) / crr;
    const float delta = -k * mr + s * Mt - c * Mn;
    const float root = sqrtf(1.0f - 4.0f * delta * k);
    const float rho = 2.0f * k / root;
    const float d = 2.0f * delta / (1.0f + root);
    float phi0 = ph + al;
    if (phi0 > kPi) phi0 -= 2.0f * kPi;
    if (phi0 <= -kPi) phi0 += 2.0f * kPi;
    // distance of each hit to the circle
    const float e = k * dr - du * s + dv * c;
    const float F = e / root;
    const float eps = 2.0f * F / (1.0f + sqrtf(1.0f + 2.0f * rho * F));
    const float chi2c = gsum(valid ? (eps / kSigmaRphi) * (eps / kSigmaRphi) : 0.0f);
    // transverse arc length from the point of closest approach d (sin phi0, -cos phi0)
    float sp, cp;
    sincosf(phi0, &sp, &cp);
    const float lx = x - d * sp, ly = y + d * cp;
    const float L = sqrtf(lx * lx + ly * ly);
    const float zz = 0.5f * fabsf(rho) * L;
    float arc;
    if (zz < 1e-3f) arc = L * (1.0f + zz * zz * (1.0f / 6.0f));
    else if (zz < 1.0f) arc = L * (asinf(zz) / zz);
    else arc = L * (0.5f * kPi / zz);
    const float sarc = valid ? ((cp * lx + sp * ly) >= 0.0f ? arc : -arc) : 0.0f;
    const float ms = gsum(sarc) * inv_n, mz = gsum(valid ? z : 0.0f) * inv_n;
    const float ds = valid ? sarc - ms : 0.0f, dz = valid ? z - mz : 0.0f;
    const float css = gsum(ds * ds), csz = gsum(ds * dz);
    const float cot = csz / css;
    const float z0 = mz - cot * ms;
    const float rz = (dz - cot * ds) / kSigmaZ;
    const float chi2l = gsum(valid ? rz * rz : 0.0f);
    // triplets: the exact circle's curvature from the compensated three-point formula
    float kappa = -rho;
    {
      // every lane takes part in the shuffles; groups of other sizes ignore the result
      const float xa = __shfl_sync(kFull, x, gbase), ya = __shfl_sync(kFull, y, gbase);
      const float xb = __shfl_sync(kFull, x, gbase + 1), yb = __shfl_sync(kFull, y, gbase + 1);
      const float xc = __shfl_sync(kFull, x, gbase + 2), yc = __shfl_sync(kFull, y, gbase + 2);
      if (n == 3) kappa = triplet_curvature(xa, ya, xb, yb, xc, yc);
    }
    if (active && sub == 0) {
      pt_track tr;
      tr.kappa = kappa;
      tr.phi0 = phi0;
      tr.d0 = d;
      tr.cot_theta = cot;
      tr.z0 = z0;
      tr.pt = 0.299792458f * bfield / (100.0f * fabsf(kappa));
      tr.chi2_circle = chi2c;
      tr.chi2_line = chi2l;
      tr.charge = kappa < 0.0f ? 1 : (kappa > 0.0f ? -1 : 0);
      tr.nhits = (uint8_t)n;
      tr.pad[0] = tr.pad[1] = 0;
      b.tracks[j] = tr;
    }
  }
}

}  // namespace

void launch_fit(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  PT_TRACE(l, s, "k_fit", k_fit<<<l.grid, 256, 0, s>>>(b, p.bfield));
}

}  // namespace ptca
