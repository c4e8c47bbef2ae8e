// Stage A3: cellular-automaton links.  Cell a = (h0, h1) is linked to cell
// b = (h1, h2) when the three hits pass the r-z alignment cut C1, the curvature cut C2
// and the beam-spot distance cut C3 (Sec. 2.2.1, Fig. 2: doublets are paired into
// triplets; the CA of Sec. 2.2.1).
//
// One thread per cell a.  Its candidates b are the cells leaving h1, stored by the
// doublet stage as up to three contiguous segments (one per outer layer of h1), each
// sorted by r-z slope t = dz/dr.  Writing t_a, t_b for the slopes of a and b, C1 reads
//   (r1-r0)(r2-r1)|t_a - t_b| <= rz0 (r2-r0) + rz1 |z2-z0|,
// and with |t_b| <= cotmax (D4) and m = the smallest r2-r1 of the segment this gives
//   |t_a - t_b| <= (rz0 + rz1 cotmax)/(r1-r0) + (rz0 + rz1 |t_a|)/m,
// a window that a binary search turns into a sub-range of the segment.  The window
// is widened by 1 % + 1e-3: float32 rounding of C1 moves its bound by at most
// ~4e-7 |t_a| (r1-r0)/m + 1e-6, below 0.1 % of the window.  Every candidate in it
// gets the exact cuts, so the window only skips pairs that cannot pass.  Segments
// that were too large to sort are scanned whole.
//
// The links of one cell are written contiguously (one warp-aggregated atomic per
// warp), which is the out-link list the ntuplet search walks.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

__global__ void __launch_bounds__(256)
    k_connect(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_cells, uint64_t cap_links) {
  const int lane = lane_id();
  const uint64_t nc = min(b.cnt[CNT_CELLS], (unsigned long long)cap_cells);
  const float wconst = fadd(cuts.rz0, fmul(cuts.rz1, cuts.cotmax));
  const int stride = gridDim.x * blockDim.x;
  for (uint64_t a0 = (uint64_t)blockIdx.x * blockDim.x; a0 < nc; a0 += stride) {
    const uint64_t a = a0 + threadIdx.x;
    const bool active = a < nc;
    uint32_t nlk = 0;
    uint32_t lb[kLocalLinks];
    float lq[kLocalLinks];
    float4 p0, p1;
    bool b0 = false;
    int L1 = 0;
    uint32_t h1 = 0;
    float ta = 0.0f;
    if (active) {
      const uint32_t h0 = b.cell_in[a];
      h1 = b.cell_out[a];
      p0 = b.hit4[h0];
      p1 = b.hit4[h1];
      b0 = ((b.hbin[h0] / B) % kLayers) == 0;
      L1 = (b.hbin[h1] / B) % kLayers;
      ta = b.cell_slope[a];
      b.best[a] = ~0ull;
    }
    // candidate scan (pass 1: count, keep the first kLocalLinks)
    auto scan = [&](bool write, uint64_t wbase) {
      uint32_t found = 0;
      const int nout = kNOuter[L1];
      for (int k = 0; k < nout; ++k) {
        const uint32_t off = b.seg_off[h1 * kMaxOuter + k];
        const uint32_t n = b.seg_cnt[h1 * kMaxOuter + k];
        if (n == 0) continue;
        const float m = b.seg_mdr[h1 * kMaxOuter + k];
        uint32_t lo = off, hi = off + n;
        float thi = __int_as_float(0x7f800000);
        if (m > 0.0f) {
          float w = (wconst / (p1.w - p0.w)) + (cuts.rz0 + cuts.rz1 * fabsf(ta)) / m;
          w = w * 1.01f + 1e-3f;
          const float tlo = ta - w;
          thi = ta + w;
          uint32_t l = lo, h = hi;  // first index with slope >= tlo
          while (l < h) {
            const uint32_t mid = (l + h) >> 1;
            if (b.cell_slope[mid] < tlo) l = mid + 1; else h = mid;
          }
          lo = l;
        }
        for (uint32_t c = lo; c < hi; ++c) {
          if (b.cell_slope[c] > thi) break;
          const float4 p2 = b.hit4[b.cell_out[c]];
          if (!link_c1(cuts, p0, p1, p2)) continue;
          float q;
          if (!link_c23(cuts, p0, b0, p1, p2, q)) continue;
          if (!write) {
            if (found < kLocalLinks) {
              lb[found] = c;
              lq[found] = q;
            }
          } else if (found >= kLocalLinks) {
            b.link_dst[wbase + found] = c;
            b.link_q[wbase + found] = q;
            b.has_in[c] = 1;
          }
          ++found;
        }
      }
      return found;
    };
    if (active) nlk = scan(false, 0);
    // warp-aggregated reservation
    const uint32_t inc = warp_incl_scan(nlk);
    const uint32_t tot = __shfl_sync(kFull, inc, 31);
    unsigned long long wbase = 0;
    if (lane == 31 && tot > 0) wbase = atomicAdd(&b.cnt[CNT_LINKS], (unsigned long long)tot);
    wbase = __shfl_sync(kFull, wbase, 31);
    if (active) {
      const uint64_t base = wbase + inc - nlk;
      if (base + nlk > cap_links) {
        atomicOr(&b.cnt[CNT_STATUS], ST_LINKS);
        b.link_off[a] = 0;
        b.link_cnt[a] = 0;
      } else {
        b.link_off[a] = (uint32_t)base;
        b.link_cnt[a] = nlk;
        const uint32_t nl = nlk < kLocalLinks ? nlk : kLocalLinks;
        for (uint32_t i = 0; i < nl; ++i) {
          b.link_dst[base + i] = lb[i];
          b.link_q[base + i] = lq[i];
          b.has_in[lb[i]] = 1;
        }
        if (nlk > kLocalLinks) scan(true, base);
      }
    }
  }
}

}  // namespace

void launch_connect(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  k_connect<<<l.grid, 256, 0, s>>>(b, p.cuts, p.phi_bins, (uint64_t)p.max_cells,
                                   (uint64_t)p.max_links);
}

}  // namespace ptca
