// Stage A2: doublets ("cells").  Every hit is paired with the hits of each adjacent
// outer layer that pass the cuts D0..D4 (Sec. 2.2.1, Fig. 2: the chain's first
// combinatorial step joins hits of neighbouring layers two by two).
//
// A warp searches the doublets of one inner hit at a time.  For each outer layer the
// candidates are the hits of the
// azimuthal window that can pass D1 and D2: a circle through the beam spot with
// curvature <= kmax turns by at most asin(kmax*ro/2) - asin(kmax*ri/2) between radii
// ri < ro, so the window is that angle (ro = the largest radius seen on the outer
// layer in this event) plus a safety margin and one bin each side.  The window is one
// contiguous range of the sorted hits (two when it wraps).  Lanes stride over it,
// test the exact float32 cuts, and stage the passing outer hits in shared memory; the
// segment is then appended with one reservation per
// (hit, outer layer), so the cells leaving a hit towards one layer are contiguous.
// Each segment records the smallest dr of its cells, which bounds the link stage's
// slope window.  Slots are reserved through a per-warp chunk allocator; unused slots
// are marked as holes.  Each cell is also counted on its outer hit, which sizes the link
// stage's per-hit lists of incoming cells.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr int kWarpsPerBlock = 8;

// Largest azimuth difference (radians) between an inner hit at ri and any outer hit
// at radius <= ro_max that can pass D1 (same hemisphere) and D2 (curvature <= kmax):
// asin(kmax*ro_max/2) - asin(kmax*ri/2), given the first term (asin_o, +inf when
// kmax*ro_max/2 >= 0.7, where only D1 bounds the angle) and the second (asin_i).
__device__ __forceinline__ float phi_window(float asin_o, float asin_i) {
  if (asin_o == __int_as_float(0x7f800000)) return kHalfPi + 1e-3f;
  return fminf(asin_o - asin_i + 1e-4f, kHalfPi + 1e-3f);
}

// Writes one cell and counts it on its outer hit (its link flags are cleared by the
// in-list scatter, which visits every cell slot).
__device__ __forceinline__ void write_cell(const Buffers& b, uint64_t c, uint32_t s, uint32_t o) {
  b.cell_in[c] = s;
  b.cell_out[c] = o;
  atomicAdd(&b.in_cnt[o], 1u);  // no return value: a fire-and-forget reduction
}

// Azimuthal window of inner hit `hi` (global bin gb) towards outer slot k: up to two
// ranges [r.x, r.y) and [r.z, r.w) of the sorted hits; all empty where the slot is
// unused or the outer layer ends inside the inner hit's radius.
__device__ __forceinline__ uint4 doublet_window(const Buffers& b, const pt_cuts& cuts, int32_t B,
                                                float bins_per_rad, uint32_t gb, float4 hi,
                                                float asin_i, int k) {
  const int el = gb / B;  // event*10 + layer
  const int e = el / kLayers, L = el - e * kLayers;
  const int bin = gb - el * B;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (k >= kNOuter[L]) return r;
  const int Lo = kOuter[L][k];
  const float ro_max = __uint_as_float(b.layer_rmax[e * kLayers + Lo]);
  if (!(ro_max > hi.w)) return r;
  const int w = (int)ceilf(phi_window(b.layer_asin[e * kLayers + Lo], asin_i) * bins_per_rad) + 1;
  const uint32_t base = (uint32_t)(e * kLayers + Lo) * (uint32_t)B;
  if (2 * w + 1 >= B) {
    r.x = b.bin_start[base];
    r.y = b.bin_start[base + B];
  } else {
    const int lo = bin - w, hb = bin + w;
    if (lo < 0) {
      r.x = b.bin_start[base + B + lo];
      r.y = b.bin_start[base + B];
      r.z = b.bin_start[base];
      r.w = b.bin_start[base + hb + 1];
    } else if (hb >= B) {
      r.x = b.bin_start[base + lo];
      r.y = b.bin_start[base + B];
      r.z = b.bin_start[base];
      r.w = b.bin_start[base + hb - B + 1];
    } else {
      r.x = b.bin_start[base + lo];
      r.y = b.bin_start[base + hb + 1];
    }
  }
  return r;
}

// Warps take chunks of 32 consecutive sorted hits from a work counter.  The chunk's
// windows are found lane-parallel (one hit per lane, all of its loads in flight at
// once) and kept in shared memory; the warp then searches them hit by hit.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 5)
    k_doublets(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_cells) {
  __shared__ uint32_t st_val[kWarpsPerBlock][kStage];
  __shared__ uint4 st_rng[kWarpsPerBlock][32][kMaxOuter];
  __shared__ float4 st_hit[kWarpsPerBlock][32];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  uint32_t* sval = st_val[wib];
  const unsigned lt_mask = (1u << lane) - 1u;

  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const float bins_per_rad = (float)B / kTwoPi;
  WarpChunk ch;
  unsigned long long used = 0;
  auto mark_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_cells);
    for (unsigned long long i = lo + lane; i < hi; i += 32) b.cell_out[i] = kHole;
  };

  for (;;) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(&b.cnt[CNT_DBL_WORK], 1ull);
    const uint64_t s0 = __shfl_sync(kFull, chunk, 0) * 32ull;
    if (s0 >= n_sorted) break;
    const uint32_t nh = (uint32_t)min((uint64_t)32, (uint64_t)n_sorted - s0);
    __syncwarp();
    if ((uint32_t)lane < nh) {
      const uint32_t s = (uint32_t)s0 + lane;
      const uint32_t gb = b.hbin[s];
      const float4 hi = b.hit4[s];
      const float asin_i = asinf(0.5f * cuts.kmax * hi.w);  // unused where the outer term is +inf
      st_hit[wib][lane] = hi;
#pragma unroll
      for (int k = 0; k < kMaxOuter; ++k)
        st_rng[wib][lane][k] = doublet_window(b, cuts, B, bins_per_rad, gb, hi, asin_i, k);
    }
    __syncwarp();

    for (uint32_t j = 0; j < nh; ++j) {
      const uint32_t s = (uint32_t)s0 + j;
      const float4 hi = st_hit[wib][j];
      for (int k = 0; k < kMaxOuter; ++k) {
        const uint4 rg = st_rng[wib][j][k];
        uint32_t cnt = 0;
        float mdr = __int_as_float(0x7f800000);
        // pass 1: test, stage up to kStage passing hits, count all
        for (int part = 0; part < 2; ++part) {
          const uint32_t beg = part ? rg.z : rg.x, end = part ? rg.w : rg.y;
          for (uint32_t o0 = beg; o0 < end; o0 += 32) {
            const uint32_t o = o0 + lane;
            bool pass = false;
            if (o < end) {
              const float4 ho = b.hit4[o];
              pass = doublet_pass(cuts, hi, ho);
              if (pass) mdr = fminf(mdr, fsub(ho.w, hi.w));
            }
            const unsigned bal = __ballot_sync(kFull, pass);
            if (pass) {
              const uint32_t pos = cnt + __popc(bal & lt_mask);
              if (pos < kStage) sval[pos] = o;
            }
            cnt += __popc(bal);
          }
        }

        uint32_t seg_off = 0, seg_cnt = 0;
        if (cnt > 0) {
          // warp minimum of dr over the passing hits
          for (int off = 16; off > 0; off >>= 1) mdr = fminf(mdr, __shfl_xor_sync(kFull, mdr, off));
          unsigned long long hlo, hhi;
          const unsigned long long base = chunk_take(ch, &b.cnt[CNT_CELLS], cnt, &hlo, &hhi);
          mark_hole(hlo, hhi);
          used += cnt;
          if (base + cnt > cap_cells) {
            if (lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_CELLS);
            mark_hole(base, base + cnt);  // slots below the capacity stay readable
          } else if (cnt <= (uint32_t)kStage) {
            __syncwarp();
            for (uint32_t i = lane; i < cnt; i += 32)
              write_cell(b, base + i, s, sval[i]);
            seg_off = (uint32_t)base;
            seg_cnt = cnt;
          } else {
            // too many for the stage: recompute and write in test order
            uint32_t pos0 = 0;
            for (int part = 0; part < 2; ++part) {
              const uint32_t beg = part ? rg.z : rg.x, end = part ? rg.w : rg.y;
              for (uint32_t o0 = beg; o0 < end; o0 += 32) {
                const uint32_t o = o0 + lane;
                bool pass = false;
                if (o < end) pass = doublet_pass(cuts, hi, b.hit4[o]);
                const unsigned bal = __ballot_sync(kFull, pass);
                if (pass) {
                  const uint64_t c = base + pos0 + __popc(bal & lt_mask);
                  write_cell(b, c, s, o);
                }
                pos0 += __popc(bal);
              }
            }
            seg_off = (uint32_t)base;
            seg_cnt = cnt;
          }
        }
        // every slot is written (empty where the layer has fewer outer layers), so
        // readers need not know the hit's layer
        if (lane == 0) {
          Segment sg;
          sg.off = seg_off;
          sg.cnt = seg_cnt;
          sg.mdr = seg_cnt ? mdr : -1.0f;
          sg.pad = 0;
          b.seg[(uint64_t)s * kMaxOuter + k] = sg;
        }
        __syncwarp();
      }
    }
  }
  mark_hole(ch.next, ch.end);
  if (lane == 0 && used) atomicAdd(&b.cnt[CNT_CELLS_USED], used);
}

}  // namespace

void launch_doublets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  cudaMemsetAsync(&b.cnt[CNT_DBL_WORK], 0, sizeof(unsigned long long), s);  // work counter
  PT_TRACE(l, s, "k_doublets",
           k_doublets<<<l.sgrid, kWarpsPerBlock * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                               (uint64_t)p.max_cells));
}

}  // namespace ptca
