// Stage A3: cellular-automaton links.  Cell a = (h0, h1) is linked to cell
// b = (h1, h2) when the three hits pass the r-z alignment cut C1, the curvature cut C2
// and the beam-spot distance cut C3 (Sec. 2.2.1, Fig. 2: doublets are paired into
// triplets by the cellular automaton).
//
// One warp per middle hit h1.  The cells leaving h1 (up to three segments, one per
// outer layer, each padded to a multiple of 8) are staged once, in one pass, in shared
// memory: their r-z slopes and the coordinates of their outer hits.  The cells ending
// on h1 come from a per-hit list of 8-byte records (cell, inner hit | inner-layer flag)
// and are taken 32 at a time, one per lane; the inner hits of the next group are
// fetched while a group is swept.  With d1 = r1-r0, d2 = r2-r1 and t_a, t_b the slopes of a and b, C1 reads
//   d1 d2 |t_a - t_b| <= rz0 (d1 + d2) + rz1 |t_a d1 + t_b d2|,
// so |t_a - t_b| <= rz0 (1/d1 + 1/d2) + rz1 (|t_a|/d2 + |t_b|/d1).  Bounding |t_b| by
// cotmax (D4), or by |t_a| + |t_a - t_b| and solving for |t_a - t_b|, and d2 by the
// smallest r2-r1 of the segment, m, gives the window
//   |t_a - t_b| <= min((rz0 + rz1 cotmax)/d1 + (rz0 + rz1 |t_a|)/m,
//                      (rz0 + rz1 |t_a|)(1/d1 + 1/m) / (1 - rz1/d1)),
// the second term only where d1 > rz1.  It is widened by 1 % + 1e-3, far beyond the
// float32 rounding of C1 (about 4e-7 |t_a| d1/m + 1e-6) and of the approximate
// quotients and reciprocals used for the slopes and the window (a few 1e-7 relative).
// The warp sweeps all staged slopes eight at a time, every lane testing its own cell
// against them with the window of the segment the eight belong to, with no divergence;
// a lane whose window holds any of the eight queues one entry (incoming index, 8-bit
// mask, position).  The queue is drained 32 entries
// at a time through the exact cuts, all lanes busy.  The links of a middle hit are
// collected in shared memory, reserved once, sorted by source cell and written as
// per-cell lists (the out-link lists the ntuplet search walks): a source's links are
// one run of equal link_src values, so the first slot of each run names a cell that
// can start an ntuplet.  If a hit has more links than the collection holds, the search
// runs a second time and writes them all to a temporary half of a double-size
// reservation, which is then sorted.  Segments larger than the stage are swept piece
// by piece.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kConnWarps = 8;
constexpr int kOutStage = 160;  // staged outgoing cells per warp (multiple of 8, < 256)
constexpr int kQueue = 128;     // candidate ring per warp (power of two, >= 31 + 32)
constexpr int kFound = 64;      // links of one group kept in shared memory (rank < 256)
constexpr uint32_t kHitChunk = 4;       // consecutive middle hits per warp chunk (<= 32)
constexpr int kScatterBlocksPerSm = 4;  // fewer warps in flight keep the scatter local
constexpr int kConnBlocksPerSm = 4;     // 64 registers per thread: no spills in the link search
static_assert(kOutStage % 8 == 0 && kOutStage < 256, "staged positions fit 8 bits");

__device__ __forceinline__ uint32_t round8(uint32_t n) { return (n + 7u) & ~7u; }

// in_rec[in_start[h] + rank] = (cell, inner hit | inner layer is 0 << 31), grouping the
// cells by the hit they end on; every cell's two link flags are cleared on the way.  One warp per inner hit, in sorted-hit order: the warps
// running at one time cover a narrow azimuthal range of a layer, so their records land
// in a narrow range of in_rec and partial sectors merge in L2 before write-back.
__global__ void k_in_scatter(Buffers b, int32_t B) {
  const int lane = lane_id();
  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const int wpb = blockDim.x >> 5;
  const int nwarps = gridDim.x * wpb;
  for (uint32_t h0 = blockIdx.x * wpb + (threadIdx.x >> 5); h0 < n_sorted; h0 += nwarps) {
    const Segment* sgp = b.seg + (uint64_t)h0 * kMaxOuter;
    const uint32_t n0 = sgp[0].cnt, n1 = sgp[1].cnt, n2 = sgp[2].cnt;
    const uint32_t n = n0 + n1 + n2;
    if (n == 0) continue;
    const uint32_t o0 = sgp[0].off, o1 = sgp[1].off, o2 = sgp[2].off;
    const uint32_t tag = h0 | ((b.hbin[h0] / (uint32_t)B) % kLayers == 0 ? 0x80000000u : 0u);
    for (uint32_t i0 = 0; i0 < n; i0 += 64) {
      uint32_t c[2], o[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t i = i0 + u * 32 + lane;
        o[u] = kHole;
        if (i < n) {
          c[u] = i < n0 ? o0 + i : (i < n0 + n1 ? o1 + (i - n0) : o2 + (i - n0 - n1));
          o[u] = b.cell_out[c[u]];

        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (o[u] != kHole) {  // the count left on the hit is the cell's slot in its list
          b.in_rec[b.in_start[o[u]] + atomicSub(&b.in_cnt[o[u]], 1u) - 1u] = make_uint2(c[u], tag);
          b.has_in[c[u]] = 0;
          b.has_out[c[u]] = 0;
        }
    }
  }
}

// Per-warp shared state.  Warp-uniform values live here rather than in registers, so
// that the sweep keeps only a lane's slope and window live.
struct ConnWarp {
  float4 p2[kOutStage];      // staged outgoing cells: outer hit
  float t[kOutStage];        //   slope (NaN padding)
  float4 p1;                 // middle hit
  Segment sg[kMaxOuter];     // outgoing segments of the middle hit
  uint32_t pos[kMaxOuter];   // staged position of each segment / piece
  uint32_t coff[kMaxOuter];  // cell of each staged position pos[k]
  unsigned long long chunk_next[1], chunk_end[1], used;  // link slots
  uint32_t chunk_size[1];
  uint32_t hin0[kHitChunk], hnin[kHitChunk];  // incoming-cell list of each hit of the chunk
  uint32_t in0, nin;         // incoming-cell list of the middle hit
  unsigned long long lbase;  // its link block
  uint32_t lvalid;           //   (within the capacity)
  uint2 q[kQueue];           // candidates: (incoming index, 8-bit mask << 8 | position)
  uint32_t fs[kFound];       // found links: source cell
  uint32_t fd[kFound];       //   target cell
  float fq[kFound];          //   quality
};

// Warp chunk reservation with the chunk state in shared memory, lane 0 acting.
__device__ __forceinline__ unsigned long long chunk_take_shared(
    ConnWarp& W, int which, unsigned long long* counter, uint32_t n, unsigned long long* hlo,
    unsigned long long* hhi) {
  unsigned long long r = 0, lo = 0, hi = 0;
  if ((threadIdx.x & 31) == 0) {
    unsigned long long next = W.chunk_next[which], end = W.chunk_end[which];
    if (next + n > end) {
      lo = next;
      hi = end;
      uint32_t size = W.chunk_size[which];
      const uint32_t want = size == 0 ? n : (n > size ? n : size);
      W.chunk_size[which] = size == 0 ? (n > kChunkMin ? n : kChunkMin) : min(2 * size, kChunkMax);
      next = atomicAdd(counter, (unsigned long long)want);
      end = next + want;
    }
    r = next;
    W.chunk_next[which] = next + n;
    W.chunk_end[which] = end;
  }
  r = __shfl_sync(kFull, r, 0);
  *hlo = __shfl_sync(kFull, lo, 0);
  *hhi = __shfl_sync(kFull, hi, 0);
  return r;
}

template <bool GATE>
__global__ void __launch_bounds__(kConnWarps * 32, kConnBlocksPerSm)
    k_connect(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_links) {
  __shared__ ConnWarp s_w[kConnWarps];
  const int lane = lane_id();
  ConnWarp& W = s_w[threadIdx.x >> 5];
  const unsigned lt_mask = (1u << lane) - 1u;
  const float kNaN = __int_as_float(0x7fc00000);
  const float kInf = __int_as_float(0x7f800000);
  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const int nwarps = gridDim.x * kConnWarps;
  if (lane == 0) {
    W.chunk_next[0] = W.chunk_end[0] = 0;
    W.chunk_size[0] = 0;
  }
  if (lane == 0) W.used = 0;
  __syncwarp();
  auto mark_link_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_links);
    for (unsigned long long i = lo + lane; i < hi; i += 32) b.link_src[i] = kHole;
  };
  auto write_link = [&](uint64_t slot, uint32_t a, uint32_t c, float q) {
    b.link_src[slot] = a;
    b.link_dst[slot] = c;
    b.link_q[slot] = q;
    if (!GATE) {  // gated form: the gate sets the flags of the links it keeps
      b.has_out[a] = 1;
      b.has_in[c] = 1;
    }
  };
  // stages cells [c0, c0 + n) leaving the middle hit p1 at position p (padded to a
  // multiple of 8 with NaN slopes); the slope only places the window, so an
  // approximate quotient is enough
  auto stage = [&](uint32_t c0, uint32_t n, uint32_t p, float4 p1) {
    for (uint32_t i = lane; i < round8(n); i += 32) {
      float t = kNaN;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < n) {
        q = b.hit4[b.cell_out[c0 + i]];
        t = __fdividef(q.z - p1.z, q.w - p1.w);
      }
      W.t[p + i] = t;
      W.p2[p + i] = q;
    }
  };

  // chunks of kHitChunk consecutive middle hits per warp; one round of loads finds the
  // hits with both incoming and outgoing cells
  for (uint32_t hc = (blockIdx.x * kConnWarps + (threadIdx.x >> 5)) * kHitChunk; hc < n_sorted;
       hc += (uint32_t)nwarps * kHitChunk) {
    bool work = false;
    {
      const uint32_t hl = hc + lane;
      uint32_t in0 = 0, nin = 0;
      if ((uint32_t)lane < kHitChunk && hl < n_sorted) {
        in0 = b.in_start[hl];
        nin = b.in_start[hl + 1] - in0;
        if (nin) {
          const Segment* sgp = b.seg + (uint64_t)hl * kMaxOuter;
          work = (sgp[0].cnt | sgp[1].cnt | sgp[2].cnt) != 0;
        }
      }
      __syncwarp();
      if ((uint32_t)lane < kHitChunk) {
        W.hin0[lane] = in0;
        W.hnin[lane] = nin;
      }
    }
    unsigned todo = __ballot_sync(kFull, work);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t h1 = hc + src;
      __syncwarp();
      if (lane == 0) {
        W.in0 = W.hin0[src];
        W.nin = W.hnin[src];
        W.lvalid = 0;
      }
      uint32_t tot = 0;
      {
        const Segment* sgp = b.seg + (uint64_t)h1 * kMaxOuter;
#pragma unroll
        for (int k = 0; k < kMaxOuter; ++k) tot += round8(sgp[k].cnt);
        __syncwarp();
        if (lane < kMaxOuter) {
          const Segment g = sgp[lane];
          W.sg[lane] = g;
          uint32_t p = 0;
          for (int k = 0; k < lane; ++k) p += round8(sgp[k].cnt);
          W.pos[lane] = p;
          W.coff[lane] = g.off;
        }
        if (lane == 0) W.p1 = b.hit4[h1];
        __syncwarp();
      }
      const bool fits = tot <= (uint32_t)kOutStage;
      // inner hit of the lane's incoming cell in the group to come: fetched ahead (the
      // first group's during the stage, each later group's during the group before), so
      // that placing a group's windows waits for one load instead of two in a row
      uint32_t h0n = (uint32_t)lane < W.nin ? (b.in_rec[W.in0 + lane].y & 0x7fffffffu) : 0u;
      if (fits) {
        // all segments in one pass over the staged positions (NaN slope for padding)
        const float4 p1 = W.p1;
        for (uint32_t P = lane; P < tot; P += 32) {
          const int k = (P >= W.pos[1]) + (P >= W.pos[2]);
          const uint32_t i = P - W.pos[k];
          float t = kNaN;
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i < W.sg[k].cnt) {
            q = b.hit4[b.cell_out[W.sg[k].off + i]];
            t = __fdividef(q.z - p1.z, q.w - p1.w);
          }
          W.t[P] = t;
          W.p2[P] = q;
        }
      }

      // Pass 0 finds the links of h1, keeps up to kFound of them in shared memory and
      // counts all; if there were more, pass 1 repeats the search and writes the rest
      // straight into the reserved block.
      uint32_t nfound = 0;
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1 && nfound <= (uint32_t)kFound) break;
        if (pass == 1)
          h0n = (uint32_t)lane < W.nin ? (b.in_rec[W.in0 + lane].y & 0x7fffffffu) : 0u;
        uint32_t head = 0, tail = 0, nf = 0;
        // exact cuts on up to 32 queued entries, all lanes busy (one round per set bit)
        auto process = [&](uint32_t nt) {
          __syncwarp();
          const bool v = (uint32_t)lane < nt;
          const uint2 e = v ? W.q[(head + lane) & (kQueue - 1)] : make_uint2(0u, 0u);
          head += nt;
          const uint32_t jb = e.y & 0xffu;
          uint32_t mask = e.y >> 8;
          uint32_t a = 0;
          float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f);
          bool qb0 = false;
          if (v) {
            const uint2 r = b.in_rec[W.in0 + e.x];
            a = r.x;
            qb0 = (r.y >> 31) != 0;
            p0 = b.hit4[r.y & 0x7fffffffu];
          }
          const float4 p1 = W.p1;
          while (__any_sync(kFull, mask != 0)) {
            bool ok = false;
            float q = 0.0f;
            uint32_t jj = 0;
            if (mask) {
              jj = jb + (__ffs(mask) - 1);
              mask &= mask - 1;
              const float4 p2 = W.p2[jj];
              ok = link_c1(cuts, p0, p1, p2) && link_c23(cuts, p0, qb0, p1, p2, q);
            }
            const unsigned pm = __ballot_sync(kFull, ok);
            if (ok) {
              const uint32_t seq = nf + __popc(pm & lt_mask);
              const int k = (jj >= W.pos[1]) + (jj >= W.pos[2]);
              const uint32_t c = W.coff[k] + (jj - W.pos[k]);
              if (pass == 0) {
                if (seq < (uint32_t)kFound) {
                  W.fs[seq] = a;
                  W.fd[seq] = c;
                  W.fq[seq] = q;
                }
              } else if (seq >= (uint32_t)kFound && W.lvalid) {
                write_link(W.lbase + nfound + seq, a, c, q);
              }
            }
            nf += __popc(pm);
          }
        };
        // sweep of staged positions [j, n) (multiples of 8) with the lane's windows w0, w1,
        // w2 for the cells of segments 0, 1, 2 (positions below pos1, below pos2, the rest;
        // a segment's positions are padded to a multiple of 8, so eight positions share
        // one window); ix = the lane's index in the incoming list.  Stops after the step
        // that brings the queue to 32 entries, or at the end; returns where it stopped.
        auto sweep = [&](uint32_t j, uint32_t n, float ta, float w0, float w1, float w2,
                         uint32_t pos1, uint32_t pos2, uint32_t ix) {
          for (; j < n; j += 8) {
            const float wk = j >= pos2 ? w2 : (j >= pos1 ? w1 : w0);
            const float4 u = *reinterpret_cast<const float4*>(&W.t[j]);
            const float4 v = *reinterpret_cast<const float4*>(&W.t[j + 4]);
            const bool c0 = fabsf(u.x - ta) <= wk, c1 = fabsf(u.y - ta) <= wk;
            const bool c2 = fabsf(u.z - ta) <= wk, c3 = fabsf(u.w - ta) <= wk;
            const bool c4 = fabsf(v.x - ta) <= wk, c5 = fabsf(v.y - ta) <= wk;
            const bool c6 = fabsf(v.z - ta) <= wk, c7 = fabsf(v.w - ta) <= wk;
            const bool any = (c0 | c1 | c2 | c3) | (c4 | c5 | c6 | c7);
            const unsigned bal = __ballot_sync(kFull, any);
            if (bal) {
              if (any) {
                const uint32_t m = (c0 ? 1u : 0u) | (c1 ? 2u : 0u) | (c2 ? 4u : 0u) | (c3 ? 8u : 0u) |
                                   (c4 ? 16u : 0u) | (c5 ? 32u : 0u) | (c6 ? 64u : 0u) |
                                   (c7 ? 128u : 0u);
                W.q[(tail + __popc(bal & lt_mask)) & (kQueue - 1)] = make_uint2(ix, (m << 8) | j);
              }
              tail += __popc(bal);
              if (tail - head >= 32u) return j + 8;
            }
          }
          return n;
        };

        for (uint32_t ib = 0; ib < W.nin; ib += 32) {
          const uint32_t ix = ib + lane;
          float ta = kNaN;
          float w[kMaxOuter];
          {
            const float4 p1 = W.p1;
            float2 zw = make_float2(0.f, 0.f);
            if (ix < W.nin) zw = *reinterpret_cast<const float2*>(&b.hit4[h0n].z);  // z, r
            h0n = ix + 32 < W.nin ? (b.in_rec[W.in0 + ix + 32].y & 0x7fffffffu) : 0u;
            if (ix < W.nin) ta = __fdividef(p1.z - zw.x, p1.w - zw.y);  // the cell's slope dz/dr
            const float id1 = __fdividef(1.0f, p1.w - zw.y);
            const float wa = (cuts.rz0 + cuts.rz1 * cuts.cotmax) * id1;
            const float ua = cuts.rz0 + cuts.rz1 * fabsf(ta);
            const float shrink = 1.0f - cuts.rz1 * id1;
#pragma unroll
            for (int k = 0; k < kMaxOuter; ++k) {
              const float m = W.sg[k].mdr;
              const float im = __fdividef(1.0f, m);
              float wk = fmaf(ua, im, wa);
              if (shrink > 0.0f) wk = fminf(wk, __fdividef(ua * (id1 + im), shrink));
              w[k] = m > 0.0f ? wk * 1.01f + 1e-3f : kInf;
            }
          }
          // One sweep site: one sweep over all staged segments, or (when they do not fit)
          // one per piece, staged in turn at position 0.  The queue is drained before a
          // stage changes and after the last sweep of h1.
          const bool last_group = ib + 32 >= W.nin;
#pragma unroll 1
          for (int k = 0; k < (fits ? 1 : kMaxOuter); ++k) {
            const uint32_t cnt = fits ? 1u : W.sg[k].cnt;
            for (uint32_t j0 = 0; j0 < cnt; j0 += kOutStage) {
              uint32_t n8 = tot, pos1 = W.pos[1], pos2 = W.pos[2];
              float w0 = w[0], w1 = w[1], w2 = w[2];
              if (!fits) {
                const uint32_t n = min(cnt - j0, (uint32_t)kOutStage);
                __syncwarp();
                stage(W.sg[k].off + j0, n, 0, W.p1);
                if (lane == 0) {
                  W.pos[0] = 0;
                  W.pos[1] = W.pos[2] = kOutStage;
                  W.coff[0] = W.sg[k].off + j0;
                }
                __syncwarp();
                n8 = round8(n);
                pos1 = pos2 = kOutStage;
                w0 = k == 0 ? w[0] : (k == 1 ? w[1] : w[2]);
              }
              const bool last = !fits || last_group;
              // one call site each for the sweep and the exact cuts (instruction cache)
              for (uint32_t j = 0;;) {
                j = sweep(j, n8, ta, w0, w1, w2, pos1, pos2, ix);
                const bool done = j >= n8;
                while (tail - head >= 32u || (done && last && tail != head))
                  process(min(32u, tail - head));
                if (done) break;
              }
            }
          }
        }
        __syncwarp();
        if (pass == 1) break;
        nfound = nf;
        if (nf == 0) break;

        // One reservation for the links of h1; with more than kFound of them, twice as
        // many slots, the second half holding them in search order until they are sorted.
        const uint32_t nres = nf <= (uint32_t)kFound ? nf : 2 * nf;
        unsigned long long hlo, hhi;
        const unsigned long long lbase = chunk_take_shared(W, 0, &b.cnt[CNT_LINKS], nres, &hlo, &hhi);
        mark_link_hole(hlo, hhi);
        const bool lvalid = lbase + nres <= cap_links;
        if (lane == 0) {
          W.used += nf;
          W.lbase = lbase;
          W.lvalid = lvalid;
        }
        if (!lvalid) {
          if (lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_LINKS);
          mark_link_hole(lbase, lbase + nres);  // slots below the capacity stay readable
        } else if (nf > (uint32_t)kFound) {
          for (uint32_t i = lane; i < (uint32_t)kFound; i += 32)
            write_link(lbase + nf + i, W.fs[i], W.fd[i], W.fq[i]);
        }
      }

      // The links of h1, sorted by source cell (stable), form one list per source:
      // link_oc (offset, count) of each source, which joins the list of possible roots.
      __syncwarp();
      if (nfound > 0 && W.lvalid) {
        const unsigned long long lbase = W.lbase;
        const bool big = nfound > (uint32_t)kFound;
        const unsigned long long tmp = lbase + nfound;  // search-order copy when big
        auto src_of = [&](uint32_t j) { return big ? b.link_src[tmp + j] : W.fs[j]; };
        for (uint32_t i0 = 0; i0 < nfound; i0 += 32) {
          const uint32_t i = i0 + lane;
          uint32_t a = kHole, rank = 0, cnt = 0, c = 0;
          float q = 0.0f;
          bool first = false;
          if (i < nfound) {
            a = src_of(i);
            first = true;
            for (uint32_t j = 0; j < nfound; ++j) {
              const uint32_t aj = src_of(j);
              rank += (aj < a) || (aj == a && j < i);
              cnt += aj == a;
              first = first && !(aj == a && j < i);
            }
            c = big ? b.link_dst[tmp + i] : W.fd[i];
            q = big ? b.link_q[tmp + i] : W.fq[i];
          }
          __syncwarp();
          if (i < nfound) {
            write_link(lbase + rank, a, c, q);
            if (first) b.link_oc[a] = make_uint2((uint32_t)(lbase + rank), cnt);
          }
        }
        if (big) {
          __syncwarp();
          mark_link_hole(tmp, tmp + nfound);
        }
      }
      __syncwarp();
    }
    __syncwarp();
  }
  __syncwarp();
  mark_link_hole(W.chunk_next[0], W.chunk_end[0]);
  if (lane == 0 && W.used) atomicAdd(&b.cnt[CNT_LINKS_USED], W.used);
}

}  // namespace

void launch_connect(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                    bool gated) {
  PT_TRACE(l, s, "scan", launch_scan(b.in_cnt, b.in_start, &b.cnt[CNT_SCAN_HITS], b.scan_part, s));
  PT_TRACE(l, s, "k_in_scatter",
           k_in_scatter<<<l.sms * kScatterBlocksPerSm, 256, 0, s>>>(b, p.phi_bins));
  if (gated)
    PT_TRACE(l, s, "k_connect",
             k_connect<true><<<l.sms * kConnBlocksPerSm, kConnWarps * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                                  (uint64_t)p.max_links));
  else
    PT_TRACE(l, s, "k_connect",
             k_connect<false><<<l.sms * kConnBlocksPerSm, kConnWarps * 32, 0, s>>>(b, p.cuts, p.phi_bins,
                                                                   (uint64_t)p.max_links));
}

}  // namespace ptca
