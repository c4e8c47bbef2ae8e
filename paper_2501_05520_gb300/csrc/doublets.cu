// Stage A2: doublets ("cells").  Every hit is paired with the hits of each adjacent
// outer layer that pass the cuts D0..D4 (Sec. 2.2.1, Fig. 2: hits in adjacent layers
// are paired to form doublets).
//
// One warp per inner hit.  For each outer layer the candidates are the hits of the
// azimuthal window that can pass D1 and D2: a circle through the beam spot with
// curvature <= kmax turns by at most asin(kmax*ro/2) - asin(kmax*ri/2) between radii
// ri < ro, so the window is that angle (ro = the largest radius seen on the outer
// layer in this event) plus a safety margin and one bin each side.  The window is one
// contiguous range of the sorted hits (two when it wraps).  Lanes stride over it,
// test the exact float32 cuts, and stage the passing outer hits in shared memory.
// The staged segment is sorted by its r-z slope dz/dr and appended with one atomic
// per (hit, outer layer), so the cells leaving a hit towards one layer are
// contiguous and slope-ordered; the link stage searches them by slope.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr int kWarpsPerBlock = 8;

// Largest azimuth difference (radians) between an inner hit at ri and any outer hit
// at radius <= ro_max that can pass D1 (same hemisphere) and D2 (curvature <= kmax).
__device__ __forceinline__ float phi_window(float kmax, float ri, float ro_max) {
  const float a = 0.5f * kmax * ro_max;
  if (a >= 0.7f) return kHalfPi + 1e-3f;  // only D1 bounds the angle
  const float b = fminf(0.5f * kmax * ri, a);
  return fminf(asinf(a) - asinf(b) + 1e-4f, kHalfPi + 1e-3f);
}

__device__ __forceinline__ void warp_sort_stage(float* key, uint32_t* val, int n) {
  const int lane = lane_id();
  int P = 32;
  while (P < n) P <<= 1;
  for (int i = n + lane; i < P; i += 32) {
    key[i] = __int_as_float(0x7f800000);  // +inf
    val[i] = 0xffffffffu;
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const float ki = key[i], kj = key[ixj];
          if ((ki > kj) == up) {
            key[i] = kj;
            key[ixj] = ki;
            const uint32_t t = val[i];
            val[i] = val[ixj];
            val[ixj] = t;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_doublets(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_cells) {
  __shared__ float st_key[kWarpsPerBlock][kStage];
  __shared__ uint32_t st_val[kWarpsPerBlock][kStage];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  float* skey = st_key[wib];
  uint32_t* sval = st_val[wib];
  const unsigned lt_mask = (1u << lane) - 1u;

  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const float bins_per_rad = (float)B / kTwoPi;
  const int nwarps = gridDim.x * kWarpsPerBlock;

  for (uint32_t s = blockIdx.x * kWarpsPerBlock + wib; s < n_sorted; s += nwarps) {
    const uint32_t gb = b.hbin[s];
    const int el = gb / B;            // event*10 + layer
    const int e = el / kLayers, L = el - e * kLayers;
    const int bin = gb - el * B;
    const float4 hi = b.hit4[s];
    const int nout = kNOuter[L];
    for (int k = 0; k < nout; ++k) {
      const int Lo = kOuter[L][k];
      const float ro_max = __uint_as_float(b.layer_rmax[e * kLayers + Lo]);
      uint32_t cnt = 0;
      float mdr = __int_as_float(0x7f800000);
      uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;  // up to two sorted-hit ranges
      if (ro_max > hi.w) {
        const int w = (int)ceilf(phi_window(cuts.kmax, hi.w, ro_max) * bins_per_rad) + 1;
        const uint32_t base = (uint32_t)(e * kLayers + Lo) * (uint32_t)B;
        if (2 * w + 1 >= B) {
          r0 = b.bin_start[base];
          r1 = b.bin_start[base + B];
        } else {
          const int lo = bin - w, hb = bin + w;
          if (lo < 0) {
            r0 = b.bin_start[base + B + lo];
            r1 = b.bin_start[base + B];
            r2 = b.bin_start[base];
            r3 = b.bin_start[base + hb + 1];
          } else if (hb >= B) {
            r0 = b.bin_start[base + lo];
            r1 = b.bin_start[base + B];
            r2 = b.bin_start[base];
            r3 = b.bin_start[base + hb - B + 1];
          } else {
            r0 = b.bin_start[base + lo];
            r1 = b.bin_start[base + hb + 1];
          }
        }
      }
      // pass 1: test, stage up to kStage passing hits, count all
      for (int part = 0; part < 2; ++part) {
        const uint32_t beg = part ? r2 : r0, end = part ? r3 : r1;
        for (uint32_t o0 = beg; o0 < end; o0 += 32) {
          const uint32_t o = o0 + lane;
          bool pass = false;
          float slope = 0.0f;
          if (o < end) {
            const float4 ho = b.hit4[o];
            pass = doublet_pass(cuts, hi, ho);
            if (pass) {
              const float dr = fsub(ho.w, hi.w);
              slope = fdiv(fsub(ho.z, hi.z), dr);
              mdr = fminf(mdr, dr);
            }
          }
          const unsigned bal = __ballot_sync(kFull, pass);
          if (pass) {
            const uint32_t pos = cnt + __popc(bal & lt_mask);
            if (pos < kStage) {
              skey[pos] = slope;
              sval[pos] = o;
            }
          }
          cnt += __popc(bal);
        }
      }
      // warp minimum of dr over the passing hits
      for (int off = 16; off > 0; off >>= 1) mdr = fminf(mdr, __shfl_xor_sync(kFull, mdr, off));

      uint32_t seg_off = 0, seg_cnt = 0;
      float seg_mdr = -1.0f;
      if (cnt > 0) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&b.cnt[CNT_CELLS], (unsigned long long)cnt);
        base = __shfl_sync(kFull, base, 0);
        if (base + cnt > cap_cells) {
          if (lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_CELLS);
        } else if (cnt <= (uint32_t)kStage) {
          __syncwarp();
          warp_sort_stage(skey, sval, (int)cnt);
          for (uint32_t i = lane; i < cnt; i += 32) {
            const uint32_t c = (uint32_t)base + i;
            b.cell_in[c] = s;
            b.cell_out[c] = sval[i];
            b.cell_slope[c] = skey[i];
            b.has_in[c] = 0;
          }
          seg_off = (uint32_t)base;
          seg_cnt = cnt;
          seg_mdr = mdr;
        } else {
          // too many for the stage: recompute and write in test order (unsorted)
          uint32_t pos0 = 0;
          for (int part = 0; part < 2; ++part) {
            const uint32_t beg = part ? r2 : r0, end = part ? r3 : r1;
            for (uint32_t o0 = beg; o0 < end; o0 += 32) {
              const uint32_t o = o0 + lane;
              bool pass = false;
              float4 ho;
              if (o < end) {
                ho = b.hit4[o];
                pass = doublet_pass(cuts, hi, ho);
              }
              const unsigned bal = __ballot_sync(kFull, pass);
              if (pass) {
                const uint32_t c = (uint32_t)base + pos0 + __popc(bal & lt_mask);
                b.cell_in[c] = s;
                b.cell_out[c] = o;
                b.cell_slope[c] = fdiv(fsub(ho.z, hi.z), fsub(ho.w, hi.w));
                b.has_in[c] = 0;
              }
              pos0 += __popc(bal);
            }
          }
          seg_off = (uint32_t)base;
          seg_cnt = cnt;
          seg_mdr = -1.0f;
        }
      }
      if (lane == 0) {
        b.seg_off[s * kMaxOuter + k] = seg_off;
        b.seg_cnt[s * kMaxOuter + k] = seg_cnt;
        b.seg_mdr[s * kMaxOuter + k] = seg_mdr;
      }
      __syncwarp();
    }
  }
}

}  // namespace

void launch_doublets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  k_doublets<<<l.sms * 8, kWarpsPerBlock * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                        (uint64_t)p.max_cells);
}

}  // namespace ptca
