// Stage A2: doublets ("cells").  Every hit is paired with the hits of each adjacent
// layer that pass the cuts D0..D4 (Sec. 2.2.1, Fig. 2: the chain's first combinatorial
// step joins hits of neighbouring layers two by two).
//
// The search runs from the outer hit of each pair towards its inner layers, so that
// the cells ending on one hit come out contiguous: for each outer hit and inner-layer
// slot, one segment of cells ordered by inner hit.  The link stage then finds the cells
// arriving at a middle hit in its own segments, with no scatter by outer hit and no
// returning atomic per cell.
//
// Candidates are the inner-layer hits of an azimuthal window that can pass D1 and D2:
// a circle through the beam spot with curvature <= kmax turns by at most
// asin(kmax*ro/2) - asin(kmax*ri/2) between radii ri < ro (and every radius of this
// detector lies on the first half of such a circle, which D1 keeps), so with ri bounded
// below by the smallest radius seen on the inner layer in this event the window is
// asin(kmax*ro/2) - asin(kmax*ri_min/2), plus a safety margin and one bin each side.
// It is one contiguous range of the sorted hits, or two when it wraps, taken in
// increasing index order.  Lanes stride over it, test the exact float32 cuts and stage
// the passing inner hits in shared memory; the segment is then appended with one
// reservation per (hit, inner slot).  Slots are reserved through a per-warp chunk
// allocator; unused slots are marked as holes.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr int kWarpsPerBlock = 8;

// Writes one cell; its two link flags start cleared.
__device__ __forceinline__ void write_cell(const Buffers& b, uint64_t c, uint32_t in, uint32_t out) {
  b.cell_in[c] = in;
  b.cell_out[c] = out;
  b.has_in[c] = 0;
  b.has_out[c] = 0;
}

// Azimuthal window of outer hit `ho` (global bin gb, asin_o = asin(kmax*ro/2), +inf where
// kmax*ro/2 >= 0.7) towards inner slot k: up to two ranges [r.x, r.y) and [r.z, r.w) of
// the sorted hits, the first below the second; empty where the slot is unused, the
// inner layer has no hit inside the outer hit's radius, or none of its r-z extent can
// pass D2 and D3 with the outer hit.
__device__ __forceinline__ uint4 reverse_window(const Buffers& b, const pt_cuts& cuts,
                                                const PairTable& pt, int32_t B,
                                                float bins_per_rad, uint32_t gb, float4 ho,
                                                float asin_o, int k) {
  const int el = gb / B;  // event*10 + layer
  const int e = el / kLayers, L = el - e * kLayers;
  const int bin = gb - el * B;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (k >= pt.n_inner[L]) return r;
  const int Li = pt.inner[L][k];
  const float ri_min = __uint_as_float(b.layer_rmin[e * kLayers + Li]);
  if (!(ho.w > ri_min)) return r;  // D0 fails for every hit of the inner layer
  if (!rz_box_reachable(cuts, ho.w, ho.z, ri_min, __uint_as_float(b.layer_rmax[e * kLayers + Li]),
                        float_from_order_key(b.layer_zmin[e * kLayers + Li]),
                        float_from_order_key(b.layer_zmax[e * kLayers + Li]), false))
    return r;
  float win = kHalfPi + 1e-3f;     // where the curvature bound is void, D1's
  if (asin_o != __int_as_float(0x7f800000))
    win = fminf(asin_o - b.layer_asin_lo[e * kLayers + Li] + 1e-4f, win);
  const int w = (int)ceilf(win * bins_per_rad) + 1;
  const uint32_t base = (uint32_t)(e * kLayers + Li) * (uint32_t)B;
  if (2 * w + 1 >= B) {
    r.x = b.bin_start[base];
    r.y = b.bin_start[base + B];
  } else {
    const int lo = bin - w, hb = bin + w;
    if (lo < 0) {
      r.x = b.bin_start[base];
      r.y = b.bin_start[base + hb + 1];
      r.z = b.bin_start[base + B + lo];
      r.w = b.bin_start[base + B];
    } else if (hb >= B) {
      r.x = b.bin_start[base];
      r.y = b.bin_start[base + hb - B + 1];
      r.z = b.bin_start[base + lo];
      r.w = b.bin_start[base + B];
    } else {
      r.x = b.bin_start[base + lo];
      r.y = b.bin_start[base + hb + 1];
    }
  }
  return r;
}

// Warps take chunks of 32 consecutive sorted (outer) hits from a work counter.  The
// chunk's windows are found lane-parallel (one hit per lane, all of its loads in flight
// at once) and kept in shared memory; the warp then searches them hit by hit.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 5)
    k_doublets(Buffers b, pt_cuts cuts, PairTable pt, int32_t B, uint64_t cap_cells) {
  __shared__ uint32_t st_val[kWarpsPerBlock][kStage];
  __shared__ uint4 st_rng[kWarpsPerBlock][32][kMaxInner];
  __shared__ float4 st_hit[kWarpsPerBlock][32];
  __shared__ uint8_t st_nin[kWarpsPerBlock][32];  // inner layers of each hit's layer
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
      const float4 ho = b.hit4[s];
      const float a = 0.5f * cuts.kmax * ho.w;
      const float asin_o = a >= 0.7f ? __int_as_float(0x7f800000) : asinf(a);
      st_hit[wib][lane] = ho;
      const int nin = pt.n_inner[(gb / (uint32_t)B) % kLayers];
      st_nin[wib][lane] = (uint8_t)nin;
      for (int k = 0; k < nin; ++k) {
        uint4 rg = reverse_window(b, cuts, pt, B, bins_per_rad, gb, ho, asin_o, k);
        if (!PT_CHECK(b.cnt, rg.x <= rg.y && rg.y <= n_sorted && rg.z <= rg.w && rg.w <= n_sorted,
                      DBG_DBL_WINDOW))
          rg = make_uint4(0u, 0u, 0u, 0u);
        st_rng[wib][lane][k] = rg;
      }
    }
    __syncwarp();

    for (uint32_t j = 0; j < nh; ++j) {
      const uint32_t s = (uint32_t)s0 + j;
      const float4 ho = st_hit[wib][j];
      const int nin = st_nin[wib][j];
      // the slots the hit's layer does not use are written empty, so readers need not
      // know the hit's layer
      if (lane >= nin && lane < pt.max_inner)
        b.seg[(uint64_t)s * pt.max_inner + lane] = make_uint2(0u, 0u);
      for (int k = 0; k < nin; ++k) {
        const uint4 rg = st_rng[wib][j][k];
        uint32_t cnt = 0;
        // pass 1: test, stage up to kStage passing hits, count all; two candidates per
        // lane in flight (both loads issued before either test)
        for (int part = 0; part < 2; ++part) {
          const uint32_t beg = part ? rg.z : rg.x, end = part ? rg.w : rg.y;
          for (uint32_t i0 = beg; i0 < end; i0 += 64) {
            float4 hv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const uint32_t i = i0 + 32 * u + lane;
              hv[u] = i < end ? b.hit4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const uint32_t i = i0 + 32 * u + lane;
              const bool pass = i < end && doublet_pass(cuts, hv[u], ho);
              const unsigned bal = __ballot_sync(kFull, pass);
              if (pass) {
                const uint32_t pos = cnt + __popc(bal & lt_mask);
                if (pos < kStage) sval[pos] = i;
              }
              cnt += __popc(bal);
            }
          }
        }

        uint32_t seg_off = 0, seg_cnt = 0;
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
            for (uint32_t i = lane; i < cnt; i += 32)
              if (PT_CHECK(b.cnt, base + i < cap_cells, DBG_DBL_CELL))
                write_cell(b, base + i, sval[i], s);
            seg_off = (uint32_t)base;
            seg_cnt = cnt;
          } else {
            // too many for the stage: recompute and write in test order
            uint32_t pos0 = 0;
            for (int part = 0; part < 2; ++part) {
              const uint32_t beg = part ? rg.z : rg.x, end = part ? rg.w : rg.y;
              for (uint32_t i0 = beg; i0 < end; i0 += 32) {
                const uint32_t i = i0 + lane;
                const bool pass = i < end && doublet_pass(cuts, b.hit4[i], ho);
                const unsigned bal = __ballot_sync(kFull, pass);
                if (pass && PT_CHECK(b.cnt, base + pos0 + __popc(bal & lt_mask) < cap_cells,
                                     DBG_DBL_CELL))
                  write_cell(b, base + pos0 + __popc(bal & lt_mask), i, s);
                pos0 += __popc(bal);
              }
            }
            seg_off = (uint32_t)base;
            seg_cnt = cnt;
          }
        }
        if (lane == 0) b.seg[(uint64_t)s * pt.max_inner + k] = make_uint2(seg_off, seg_cnt);
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
           k_doublets<<<l.sgrid, kWarpsPerBlock * 32, 0, s>>>(b, p.cuts, p.pairs, p.phi_bins,
                                                               (uint64_t)p.max_cells));
}

}  // namespace ptca
