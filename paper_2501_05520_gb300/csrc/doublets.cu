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
// The staged segment is sorted by its r-z slope dz/dr and appended with one atomic per
// (hit, outer layer), so the cells leaving a hit towards one layer are contiguous and
// slope-ordered; the link stage searches them by slope.  Slots are reserved through a
// per-warp chunk allocator; unused slots are marked as holes.  The sort runs on single
// 32-bit keys in registers (bitonic network over the warp): the order-preserving bits
// of the slope with the low 8 bits replaced by the staging position, which both makes
// the keys unique and locates the outer hit after sorting.  Each cell also takes its
// rank among the cells ending on its outer hit, from which the link stage's per-hit
// lists of incoming cells are built.
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

// Bitonic sort of 32*E unique uint32 keys held in registers, element i = e*32 + lane,
// ascending.  Partners closer than 32 elements are exchanged with xor shuffles, farther
// ones live in the same lane.
template <int E>
__device__ __forceinline__ void warp_bitonic(uint32_t (&k)[E]) {
  const int lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = e ^ (j >> 5);
          if (p > e) {
            const bool up = ((e * 32 + lane) & size) == 0;
            const uint32_t lo = min(k[e], k[p]), hi = max(k[e], k[p]);
            k[e] = up ? lo : hi;
            k[p] = up ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t o = __shfl_xor_sync(kFull, k[e], j);
          const bool up = ((e * 32 + lane) & size) == 0;
          const bool lower = (lane & j) == 0;
          k[e] = (lower == up) ? min(k[e], o) : max(k[e], o);
        }
      }
    }
  }
}

// Writes one cell and takes its rank among the cells ending on the same outer hit.
__device__ __forceinline__ void write_cell(const Buffers& b, uint64_t c, uint32_t s, uint32_t o,
                                          uint32_t key, uint8_t L) {
  b.cell_in[c] = s;
  b.cell_out[c] = o;
  b.cell_key[c] = key;
  b.cell_l0[c] = L;
  b.has_in[c] = 0;
  b.has_out[c] = 0;
  b.cell_inrank[c] = atomicAdd(&b.in_cnt[o], 1u);
}

// Sorts the n staged keys (slope bits | staging position) and writes the cells
// base..base+n in key order.
template <int E>
__device__ __forceinline__ void sort_and_write(const Buffers& b, const uint32_t* skey,
                                               const uint32_t* sval, uint32_t n, uint64_t base,
                                               uint32_t s, uint8_t L) {
  const int lane = lane_id();
  uint32_t k[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = e * 32 + lane;
    k[e] = i < n ? skey[i] : 0xffffffffu;
  }
  warp_bitonic<E>(k);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = e * 32 + lane;
    if (i < n) write_cell(b, base + i, s, sval[k[e] & 0xffu], k[e], L);
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, 5)
    k_doublets(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_cells) {
  __shared__ uint32_t st_key[kWarpsPerBlock][kStage];
  __shared__ uint32_t st_val[kWarpsPerBlock][kStage];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  uint32_t* skey = st_key[wib];
  uint32_t* sval = st_val[wib];
  const unsigned lt_mask = (1u << lane) - 1u;

  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const float bins_per_rad = (float)B / kTwoPi;
  const int nwarps = gridDim.x * kWarpsPerBlock;
  WarpChunk ch;
  unsigned long long used = 0;
  auto mark_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_cells);
    for (unsigned long long i = lo + lane; i < hi; i += 32) {
      b.cell_out[i] = kHole;
      b.has_in[i] = 0;
      b.has_out[i] = 0;
    }
  };

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
              skey[pos] = (f2ord(slope) & kKeyMask) | pos;
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
        unsigned long long hlo, hhi;
        const unsigned long long base = chunk_take(ch, &b.cnt[CNT_CELLS], cnt, &hlo, &hhi);
        mark_hole(hlo, hhi);
        used += cnt;
        if (base + cnt > cap_cells) {
          if (lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_CELLS);
          mark_hole(base, base + cnt);  // slots below the capacity stay readable
        } else if (cnt <= (uint32_t)kStage) {
          __syncwarp();
          if (cnt <= 32) sort_and_write<1>(b, skey, sval, cnt, base, s, (uint8_t)L);
          else if (cnt <= 64) sort_and_write<2>(b, skey, sval, cnt, base, s, (uint8_t)L);
          else if (cnt <= 128) sort_and_write<4>(b, skey, sval, cnt, base, s, (uint8_t)L);
          else sort_and_write<8>(b, skey, sval, cnt, base, s, (uint8_t)L);
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
                const uint64_t c = base + pos0 + __popc(bal & lt_mask);
                write_cell(b, c, s, o,
                           f2ord(fdiv(fsub(ho.z, hi.z), fsub(ho.w, hi.w))) & kKeyMask,
                           (uint8_t)L);
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
        Segment sg;
        sg.off = seg_off;
        sg.cnt = seg_cnt;
        sg.mdr = seg_mdr;
        sg.pad = 0;
        b.seg[s * kMaxOuter + k] = sg;
      }
      __syncwarp();
    }
    // unused slots of this hit's layer are empty, so readers need not know the layer
    if (lane < kMaxOuter && lane >= nout) {
      Segment sg;
      sg.off = 0;
      sg.cnt = 0;
      sg.mdr = -1.0f;
      sg.pad = 0;
      b.seg[s * kMaxOuter + lane] = sg;
    }
  }
  mark_hole(ch.next, ch.end);
  if (lane == 0 && used) atomicAdd(&b.cnt[CNT_CELLS_USED], used);
}

}  // namespace

void launch_doublets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  k_doublets<<<l.sgrid, kWarpsPerBlock * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                        (uint64_t)p.max_cells);
}

}  // namespace ptca
