// Stage A3: cellular-automaton links.  Cell a = (h0, h1) is linked to cell
// b = (h1, h2) when the three hits pass the r-z alignment cut C1, the curvature cut C2
// and the beam-spot distance cut C3 (Sec. 2.2.1, Fig. 2: doublets are paired into
// triplets by the cellular automaton).
//
// One warp per middle hit h1.  The cells leaving h1 (up to three segments, one per
// outer layer, each sorted by r-z slope) are staged once in shared memory with the
// coordinates of their outer hits; the cells ending on h1 (grouped by the ranks the
// doublet stage took) are spread over the lanes.  Writing t_a, t_b for the slopes of a
// and b, C1 reads
//   (r1-r0)(r2-r1)|t_a - t_b| <= rz0 (r2-r0) + rz1 |z2-z0|,
// and with |t_b| <= cotmax (D4) and m = the smallest r2-r1 of the segment this gives
//   |t_a - t_b| <= (rz0 + rz1 cotmax)/(r1-r0) + (rz0 + rz1 |t_a|)/m,
// a window that a binary search over the staged slope keys turns into a sub-range.
// The window is widened by 1 % + 1e-3: float32 rounding of C1 moves its bound by at
// most ~4e-7 |t_a| (r1-r0)/m + 1e-6 and the 8 dropped key bits move a slope by at most
// 3e-5 relative, both far inside the margin.  Every candidate in the window gets the
// exact cuts, so the window only skips pairs that cannot pass.  Segments that were too
// large to sort are scanned whole.
//
// The links of one cell are written contiguously (one warp-aggregated atomic per
// warp), which is the out-link list the ntuplet search walks; cells with at least one
// link are appended to a compact list, the only cells that can start an ntuplet.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kConnWarps = 8;
constexpr int kOutStage = 224;  // staged outgoing cells per warp

// in_list[in_start[h] + rank] = cell, grouping the cells by the hit they end on.
__global__ void k_in_scatter(Buffers b, uint64_t cap_cells) {
  const uint64_t nc = min(b.cnt[CNT_CELLS], (unsigned long long)cap_cells);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
    const uint32_t o = b.cell_out[c];
    if (o != kHole) b.in_list[b.in_start[o] + b.cell_inrank[c]] = (uint32_t)c;
  }
}

template <bool GATE>
__global__ void __launch_bounds__(kConnWarps * 32, 5)
    k_connect(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_links) {
  __shared__ float4 st_p2[kConnWarps][kOutStage];
  __shared__ uint32_t st_key[kConnWarps][kOutStage];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  float4* sp2 = st_p2[wib];
  uint32_t* skey = st_key[wib];
  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const float wconst = fadd(cuts.rz0, fmul(cuts.rz1, cuts.cotmax));
  const int nwarps = gridDim.x * kConnWarps;
  WarpChunk lch, kch;  // link slots, root-candidate slots
  unsigned long long used = 0;
  auto mark_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_links);
    for (unsigned long long i = lo + lane; i < hi; i += 32) b.lk_cells[i] = kHole;
  };
  auto mark_link_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_links);
    for (unsigned long long i = lo + lane; i < hi; i += 32) b.link_src[i] = kHole;
  };

  for (uint32_t h1 = blockIdx.x * kConnWarps + wib; h1 < n_sorted; h1 += nwarps) {
    const uint32_t in0 = b.in_start[h1], nin = b.in_start[h1 + 1] - in0;
    if (nin == 0) continue;
    Segment sg[kMaxOuter];
    uint32_t sbase[kMaxOuter];
    uint32_t nout = 0;
#pragma unroll
    for (int k = 0; k < kMaxOuter; ++k) {
      sg[k] = b.seg[(uint64_t)h1 * kMaxOuter + k];
      sbase[k] = nout;
      nout += sg[k].cnt;
    }
    if (nout == 0) continue;
    const bool staged = nout <= (uint32_t)kOutStage;
    if (staged) {
      for (uint32_t i = lane; i < nout; i += 32) {
        const int k = i < sbase[1] ? 0 : (i < sbase[2] ? 1 : 2);
        const uint32_t c = sg[k].off + (i - sbase[k]);
        skey[i] = b.cell_key[c];
        sp2[i] = b.hit4[b.cell_out[c]];
      }
    }
    __syncwarp();
    const float4 p1 = b.hit4[h1];

    for (uint32_t ib = 0; ib < nin; ib += 32) {
      const bool active = ib + lane < nin;
      uint32_t a = 0, nlk = 0;
      uint32_t lb[kLocalLinks];
      float lq[kLocalLinks];
      float4 p0;
      bool b0 = false;
      float ta = 0.0f;
      if (active) {
        a = b.in_list[in0 + ib + lane];
        p0 = b.hit4[b.cell_in[a]];
        ta = ord2f(b.cell_key[a] & kKeyMask);
        b0 = b.cell_l0[a] == 0;
      }
      // write == false: count, keep the first kLocalLinks in registers;
      // write == true: store the links beyond the first kLocalLinks at wbase + index
      auto scan = [&](bool write, uint64_t wbase) {
        uint32_t found = 0;
        const float inv_dr01 = 1.0f / (p1.w - p0.w);
#pragma unroll 1
        for (int k = 0; k < kMaxOuter; ++k) {
          const uint32_t n = sg[k].cnt;
          if (n == 0) continue;
          uint32_t lo = 0;
          uint32_t khi = 0xffffffffu;
          if (sg[k].mdr > 0.0f) {
            float w = wconst * inv_dr01 + (cuts.rz0 + cuts.rz1 * fabsf(ta)) / sg[k].mdr;
            w = w * 1.01f + 1e-3f;
            const uint32_t klo = f2ord(ta - w) & kKeyMask;
            khi = f2ord(ta + w) | ~kKeyMask;
            uint32_t h = n;  // first index whose key is >= klo
            while (lo < h) {
              const uint32_t mid = (lo + h) >> 1;
              const uint32_t km = staged ? skey[sbase[k] + mid] : b.cell_key[sg[k].off + mid];
              if (km < klo) lo = mid + 1; else h = mid;
            }
          }
          for (uint32_t j = lo; j < n; ++j) {
            float4 p2;
            if (staged) {
              if (skey[sbase[k] + j] > khi) break;
              p2 = sp2[sbase[k] + j];
            } else {
              if (b.cell_key[sg[k].off + j] > khi) break;
              p2 = b.hit4[b.cell_out[sg[k].off + j]];
            }
            if (!link_c1(cuts, p0, p1, p2)) continue;
            float q;
            if (!link_c23(cuts, p0, b0, p1, p2, q)) continue;
            const uint32_t c = sg[k].off + j;
            if (!write) {
              if (found < kLocalLinks) {
                lb[found] = c;
                lq[found] = q;
              }
            } else if (found >= kLocalLinks) {
              b.link_dst[wbase + found] = c;
              b.link_q[wbase + found] = q;
              if (GATE) b.link_src[wbase + found] = a;
              else b.has_in[c] = 1;
            }
            ++found;
          }
        }
        return found;
      };
      if (active) nlk = scan(false, 0);
      // warp-aggregated reservation of the link slots and of the root-candidate list
      const uint32_t inc = warp_incl_scan(nlk);
      const uint32_t tot = __shfl_sync(kFull, inc, 31);
      const unsigned has = __ballot_sync(kFull, nlk > 0);
      unsigned long long wbase = 0, lbase = 0;
      if (tot > 0) {
        unsigned long long hlo, hhi;
        wbase = chunk_take(lch, &b.cnt[CNT_LINKS], tot, &hlo, &hhi);
        if (GATE) mark_link_hole(hlo, hhi);
        lbase = chunk_take(kch, &b.cnt[CNT_LKCELLS], __popc(has), &hlo, &hhi);
        mark_hole(hlo, hhi);
        used += tot;
      }
      if (active && nlk > 0) {
        const uint64_t base = wbase + inc - nlk;
        const uint64_t li = lbase + __popc(has & lt_mask);
        if (base + nlk > cap_links || li >= cap_links) {
          atomicOr(&b.cnt[CNT_STATUS], ST_LINKS);
          if (li < cap_links) b.lk_cells[li] = kHole;  // keep the list readable
          if (GATE)
            for (uint64_t i = base; i < base + nlk && i < cap_links; ++i) b.link_src[i] = kHole;
        } else {
          b.link_off[a] = (uint32_t)base;
          b.link_cnt[a] = nlk;
          if (!GATE) b.has_out[a] = 1;  // gated form: set by the gate for kept links
          b.lk_cells[li] = a;
          const uint32_t nl = nlk < kLocalLinks ? nlk : kLocalLinks;
          for (uint32_t i = 0; i < nl; ++i) {
            b.link_dst[base + i] = lb[i];
            b.link_q[base + i] = lq[i];
            if (GATE) b.link_src[base + i] = a;
            else b.has_in[lb[i]] = 1;
          }
          if (nlk > kLocalLinks) scan(true, base);
        }
      }
    }
    __syncwarp();
  }
  mark_hole(kch.next, kch.end);
  if (GATE) mark_link_hole(lch.next, lch.end);
  if (lane == 0 && used) atomicAdd(&b.cnt[CNT_LINKS_USED], used);
}

}  // namespace

void launch_connect(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                    bool gated) {
  launch_scan(b.in_cnt, b.in_start, &b.cnt[CNT_SCAN_HITS], b.scan_part, s);
  k_in_scatter<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_cells);
  if (gated)
    k_connect<true><<<l.sgrid, kConnWarps * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                          (uint64_t)p.max_links);
  else
    k_connect<false><<<l.sgrid, kConnWarps * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                           (uint64_t)p.max_links);
}

}  // namespace ptca
