// Stage A3: cellular-automaton links.  Cell a = (h0, h1) is linked to cell
// b = (h1, h2) when the three hits pass the r-z alignment cut C1, the curvature cut C2
// and the beam-spot distance cut C3 (Sec. 2.2.1, Fig. 2: doublets are paired into
// triplets by the cellular automaton).
//
// One warp per middle hit h1.  The cells arriving at h1 are its incoming segments
// (written contiguously by the doublet stage).  The cells leaving h1 are found again
// here by the doublet search towards its outer layers (the same window and exact cuts,
// so exactly the cells the doublet stage made), staged in shared memory with their
// outer hit and r-z slope, and ordered by slope with a counting sort into 128 buckets
// spanning the staged slopes.  With d1 = r1-r0, d2 = r2-r1 and t_a, t_b the slopes of
// a and b, C1 reads
//   d1 d2 |t_a - t_b| <= rz0 (d1 + d2) + rz1 |t_a d1 + t_b d2|,
// so |t_a - t_b| <= rz0 (1/d1 + 1/d2) + rz1 (|t_a|/d2 + |t_b|/d1).  Bounding |t_b| by
// cotmax (D4), or by |t_a| + |t_a - t_b| and solving for |t_a - t_b|, and d2 by the
// smallest r2-r1 of the staged cells, m, gives the window
//   |t_a - t_b| <= min((rz0 + rz1 cotmax)/d1 + (rz0 + rz1 |t_a|)/m,
//                      (rz0 + rz1 |t_a|)(1/d1 + 1/m) / (1 - rz1/d1)),
// the second term only where d1 > rz1.  It is widened by 1 % + 1e-3, far beyond the
// float32 rounding of C1 (about 4e-7 |t_a| d1/m + 1e-6) and of the approximate
// quotients used for the slopes and the window (a few 1e-7 relative).  Each lane takes
// one incoming cell and visits only the buckets its window overlaps (the bucket of a
// slope is a monotone function of it, evaluated the same way for the staged slopes and
// for the window's ends, which are moved out by a further 0.1 % + 1e-5 so that rounding
// of t_a -+ w cannot exclude a bucket); the staged cells there that fall inside the
// window are queued as (source cell, target) pairs.  A queued pair carries all it needs,
// so the queue runs on across incoming groups and middle hits, and C1, C2 and C3 are
// tested only once 32 pairs are waiting, all lanes busy (about six pairs fall in the
// windows of a group of 32 incoming cells).  A link takes the next slot of the warp's
// reservation and is pushed onto its source's out-link list (cell_head, link_next),
// the list the ntuplet search walks; a cell's list head is cleared by the lane that
// holds the cell before any of its pairs is queued.
//
// The target cell (h1, h2) of a link is found afterwards, one thread per link, in h2's
// incoming segment from h1's layer (ordered by inner hit) by binary search: in the
// warp's own path those dependent loads would hold up the search.  A middle hit with
// more outgoing cells than the stage holds is handled piece by piece, every incoming
// group visiting every piece.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr int kConnWarps = 8;
constexpr int kConnBlocksPerSm = 4;  // 64 registers per thread
constexpr int kOut = 128;            // staged outgoing cells of one piece (<= 256)
constexpr int kNb = 128;             // slope buckets of a piece (a multiple of 32)
static_assert(kNb % 32 == 0, "buckets are scanned kNb / 32 per lane");
constexpr int kQueue = 64;           // window pairs waiting for C1-C3 (power of two)
static_assert(kOut <= 256 && kOut % 32 == 0, "staged index fits 8 bits");
static_assert(kQueue >= 63 && (kQueue & (kQueue - 1)) == 0, "queue holds 31 + 32 entries");

// Azimuthal window of inner hit `hi` (global bin gb, asin_i = asin(kmax*ri/2)) towards
// outer slot k, the doublet search's window from the inner side: the outer layer's
// asin(kmax*ro_max/2) - asin_i (+1e-4 rad, +1 bin); up to two ranges [r.x, r.y) and
// [r.z, r.w) of the sorted hits; empty where the slot is unused, the outer layer ends
// inside the inner hit's radius, or none of its r-z extent can pass D2 and D3 with the
// inner hit.
__device__ __forceinline__ uint4 forward_window(const Buffers& b, const pt_cuts& cuts,
                                                const PairTable& pt, int32_t B,
                                                float bins_per_rad, uint32_t gb, float4 hi,
                                                float asin_i, int k) {
  const int el = gb / B;  // event*10 + layer
  const int e = el / kLayers, L = el - e * kLayers;
  const int bin = gb - el * B;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (k >= pt.n_outer[L]) return r;
  const int Lo = pt.outer[L][k];
  const float ro_max = __uint_as_float(b.layer_rmax[e * kLayers + Lo]);
  if (!(ro_max > hi.w)) return r;
  if (!rz_box_reachable(cuts, hi.w, hi.z, __uint_as_float(b.layer_rmin[e * kLayers + Lo]), ro_max,
                        float_from_order_key(b.layer_zmin[e * kLayers + Lo]),
                        float_from_order_key(b.layer_zmax[e * kLayers + Lo]), true))
    return r;
  const float asin_o = b.layer_asin[e * kLayers + Lo];
  float win = kHalfPi + 1e-3f;
  if (asin_o != __int_as_float(0x7f800000)) win = fminf(asin_o - asin_i + 1e-4f, win);
  const int w = (int)ceilf(win * bins_per_rad) + 1;
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

// Per-warp shared state.
struct ConnWarp {
  float t[kOut];             // staged outgoing cells: r-z slope
  uint32_t code[kOut];       //   outer hit (sorted index) | slot of the middle hit's layer
                             //   among the outer hit's inner layers << 29
  uint8_t perm[kOut];        // bucket order -> staged index
  float ts[kOut];            // slopes in bucket order
  uint32_t bstart[kNb + 1];  // first bucket-ordered position of each slope bucket
  float4 qp0[kQueue];        // window pairs: the source's inner hit (x, y, z, r)
  uint4 q[kQueue];           //   source cell, target (outer hit | slot << 29), middle hit,
                             //   inner hit on layer 0
  float4 p1;                 // middle hit
  uint4 rg[kMaxOuter];       //   its forward windows, one per outer slot
  uint32_t so[kMaxInner];    //   its incoming segments: first cell
  uint32_t sc[kMaxInner];    //   and number of cells
  uint32_t sb[kMaxInner + 1];  //   incoming cells before each segment (the last: all)
  float tmin, scale, m;      // the staged piece: slope origin and scale of the buckets,
                             //   smallest r2 - r1
  int piece;                 // the staged piece (-1: none)
  unsigned long long chunk_next, chunk_end, used;  // link slots
  uint32_t chunk_size;
};

// Bucket of a slope (monotone non-decreasing in x): the same correctly rounded
// operations for the staged slopes and the window ends.
__device__ __forceinline__ int slope_bucket(float x, float tmin, float scale) {
  const int k = __float2int_rz(__fmul_rn(__fsub_rn(x, tmin), scale));
  return min(kNb - 1, max(0, k));
}

// Largest chunk of link slots a warp takes at once: a warp's last chunk is mostly
// unused (a hole), and link slots are scanned by the later stages.
constexpr uint32_t kLinkChunkMax = 256;

// Warp chunk reservation with the chunk state in shared memory, lane 0 acting.
__device__ __forceinline__ unsigned long long chunk_take_shared(
    ConnWarp& W, unsigned long long* counter, uint32_t n, unsigned long long* hlo,
    unsigned long long* hhi) {
  unsigned long long r = 0, lo = 0, hi = 0;
  if ((threadIdx.x & 31) == 0) {
    unsigned long long next = W.chunk_next, end = W.chunk_end;
    if (next + n > end) {
      lo = next;
      hi = end;
      const uint32_t size = W.chunk_size;
      const uint32_t want = size == 0 ? n : (n > size ? n : size);
      W.chunk_size = size == 0 ? (n > kChunkMin ? n : kChunkMin) : min(2 * size, kLinkChunkMax);
      next = atomicAdd(counter, (unsigned long long)want);
      end = next + want;
    }
    r = next;
    W.chunk_next = next + n;
    W.chunk_end = end;
  }
  r = __shfl_sync(kFull, r, 0);
  *hlo = __shfl_sync(kFull, lo, 0);
  *hhi = __shfl_sync(kFull, hi, 0);
  return r;
}

template <bool GATE>
__global__ void __launch_bounds__(kConnWarps * 32, kConnBlocksPerSm)
    k_connect(Buffers b, pt_cuts cuts, PairTable pt, int32_t B, uint64_t cap_links) {
  __shared__ ConnWarp s_w[kConnWarps];
  const int lane = lane_id();
  ConnWarp& W = s_w[threadIdx.x >> 5];
  const unsigned lt_mask = (1u << lane) - 1u;
  const int E = b.hdr->n_events;
  const uint32_t n_sorted = b.bin_start[E * kLayers * B];
  const float bins_per_rad = (float)B / kTwoPi;
  if (lane == 0) {
    W.chunk_next = W.chunk_end = 0;
    W.chunk_size = 0;
    W.used = 0;
  }
  __syncwarp();
  auto mark_link_hole = [&](unsigned long long lo, unsigned long long hi) {
    hi = min(hi, (unsigned long long)cap_links);
    for (unsigned long long i = lo + lane; i < hi; i += 32) b.link_src[i] = kHole;
  };
  // C1, C2 and C3 on nt queued pairs, one per lane, all of them carrying what they need
  // (the source cell and the target's outer hit and slot), so that pairs of different
  // incoming groups and middle hits share one pass; a link is appended to its source's
  // out-link list.
  uint32_t qhead = 0, qtail = 0;  // warp-uniform queue positions
  auto process = [&](uint32_t nt) {
    __syncwarp();
    const bool v = (uint32_t)lane < nt;
    const uint32_t qi = (qhead + lane) & (kQueue - 1);
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v) {
      e = W.q[qi];
      q0 = W.qp0[qi];
    }
    qhead += nt;
    __syncwarp();
    bool ok = false;
    float q = 0.0f;
    const uint32_t src = e.x;
    if (v) {
      const float4 q1 = b.hit4[e.z], q2 = b.hit4[e.y & 0x1fffffffu];
      ok = link_c1(cuts, q0, q1, q2) && link_c23(cuts, q0, e.w != 0, q1, q2, q);
    }
    const unsigned pm = __ballot_sync(kFull, ok);
    const uint32_t n = __popc(pm);
    if (n) {
      unsigned long long hlo, hhi;
      const unsigned long long base = chunk_take_shared(W, &b.cnt[CNT_LINKS], n, &hlo, &hhi);
      mark_link_hole(hlo, hhi);
      if (lane == 0) W.used += n;
      if (base + n > cap_links) {
        if (lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_LINKS);
        mark_link_hole(base, base + n);  // slots below the capacity stay readable
      } else if (ok) {
        const uint64_t slot = base + __popc(pm & lt_mask);
        if (PT_CHECK(b.cnt, slot < cap_links, DBG_CON_LINK)) {
          b.link_src[slot] = src;
          b.link_dst[slot] = e.y;  // outer hit | slot << 29, made a cell id by k_link_targets
          b.link_q[slot] = q;
          b.link_next[slot] = atomicExch(&b.cell_head[src], (uint32_t)slot);
          if (!GATE) b.has_out[src] = 1;  // gated form: the gate sets the flags of kept links
        }
      }
    }
    __syncwarp();
  };

  for (;;) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(&b.cnt[CNT_LNK_WORK], 1ull);
    const uint64_t s0 = __shfl_sync(kFull, chunk, 0) * 32ull;
    if (s0 >= n_sorted) break;
    // one round of loads finds the hits with incoming cells and outer layers
    uint32_t my_gb = 0;
    bool work = false;
    {
      const uint64_t s = s0 + lane;
      if (s < n_sorted) {
        my_gb = b.hbin[s];
        const int L = (my_gb / (uint32_t)B) % kLayers;
        if (pt.n_outer[L] > 0) {
          uint32_t any = 0;
          // slots past the layer's own inner layers are written empty
          for (int k = 0; k < pt.n_inner[L]; ++k) any |= b.seg[s * pt.max_inner + k].y;
          work = any != 0;
        }
      }
    }
    unsigned todo = __ballot_sync(kFull, work);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t h1 = (uint32_t)s0 + src;
      const uint32_t gb = __shfl_sync(kFull, my_gb, src);
      const int L1 = (gb / (uint32_t)B) % kLayers;
      const float4 p1 = b.hit4[h1];
      __syncwarp();
      {
        // h1's incoming segments, one slot per lane, and the cells before each
        const uint2 sgl = lane < pt.n_inner[L1] ? b.seg[(uint64_t)h1 * pt.max_inner + lane]
                                              : make_uint2(0u, 0u);
        const uint32_t inc = warp_incl_scan(sgl.y);
        if (lane < kMaxInner) {
          W.so[lane] = sgl.x;
          W.sc[lane] = sgl.y;
          W.sb[lane] = inc - sgl.y;
        }
        if (lane == kMaxInner) W.sb[kMaxInner] = inc;
      }
      // forward windows, one outer slot per lane
      if (lane < kMaxOuter) {
        uint4 rg = forward_window(b, cuts, pt, B, bins_per_rad, gb, p1,
                                  asinf(0.5f * cuts.kmax * p1.w), lane);
        if (!PT_CHECK(b.cnt, rg.x <= rg.y && rg.y <= n_sorted && rg.z <= rg.w && rg.w <= n_sorted,
                      DBG_CON_WINDOW))
          rg = make_uint4(0u, 0u, 0u, 0u);
        W.rg[lane] = rg;
      }
      if (lane == 0) {
        W.p1 = p1;
        W.piece = -1;
      }
      __syncwarp();
      const uint32_t nin = W.sb[kMaxInner];

      // Stages piece `piece` (the passing outgoing cells of ordinal [piece*kOut,
      // (piece+1)*kOut) in search order) and orders it by slope; returns the number of
      // outgoing cells of h1.
      auto stage_piece = [&](int piece) -> uint32_t {
        const uint32_t lo_ord = (uint32_t)piece * kOut;
        uint32_t cnt = 0;
        float m = __int_as_float(0x7f800000), tlo = m, thi = -m;
        for (int k = 0; k < pt.n_outer[L1]; ++k) {
          const uint8_t j2 = (uint8_t)pt.slot[pt.outer[L1][k]][L1];
          for (int part = 0; part < 2; ++part) {
            const uint4 rk = W.rg[k];
            const uint32_t beg = part ? rk.z : rk.x, end = part ? rk.w : rk.y;
            // two candidates per lane in flight: both loads are issued before either test
            for (uint32_t o0 = beg; o0 < end; o0 += 64) {
              float4 hv[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const uint32_t o = o0 + 32 * u + lane;
                hv[u] = o < end ? b.hit4[o] : make_float4(0.f, 0.f, 0.f, 0.f);
              }
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const uint32_t o = o0 + 32 * u + lane;
                const float4 ho = hv[u];
                const bool pass = o < end && doublet_pass(cuts, p1, ho);
                const unsigned bal = __ballot_sync(kFull, pass);
                if (pass) {
                  const uint32_t pos = cnt + __popc(bal & lt_mask);
                  if (pos >= lo_ord && pos < lo_ord + kOut) {
                    const uint32_t st = pos - lo_ord;
                    const float t = __fdividef(ho.z - p1.z, ho.w - p1.w);
                    W.t[st] = t;
                    W.code[st] = o | ((uint32_t)j2 << 29);
                    m = fminf(m, fsub(ho.w, p1.w));
                    tlo = fminf(tlo, t);
                    thi = fmaxf(thi, t);
                  }
                }
                cnt += __popc(bal);
              }
            }
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          m = fminf(m, __shfl_xor_sync(kFull, m, off));
          tlo = fminf(tlo, __shfl_xor_sync(kFull, tlo, off));
          thi = fmaxf(thi, __shfl_xor_sync(kFull, thi, off));
        }
        const uint32_t n = cnt > lo_ord ? min(cnt - lo_ord, (uint32_t)kOut) : 0u;
        const float scale = thi - tlo > 1e-6f ? __fdiv_rn((float)kNb, thi - tlo) : 0.0f;
        // counting sort of the staged cells by slope bucket
        __syncwarp();
        for (int i = lane; i <= kNb; i += 32) W.bstart[i] = 0;
        __syncwarp();
        int key[kOut / 32];
        uint32_t rank[kOut / 32];
#pragma unroll
        for (int u = 0; u < kOut / 32; ++u) {
          const uint32_t st = lane + 32 * u;
          key[u] = 0;
          rank[u] = 0;
          if (st < n) {
            key[u] = slope_bucket(W.t[st], tlo, scale);
            rank[u] = atomicAdd(&W.bstart[key[u] + 1], 1u);
          }
        }
        __syncwarp();
        {
          // bucket starts: kNb / 32 consecutive buckets per lane
          uint32_t cb[kNb / 32], sum = 0;
#pragma unroll
          for (int u = 0; u < kNb / 32; ++u) {
            cb[u] = W.bstart[(kNb / 32) * lane + u + 1];
            sum += cb[u];
          }
          uint32_t run = warp_incl_scan(sum) - sum;
          __syncwarp();
#pragma unroll
          for (int u = 0; u < kNb / 32; ++u) {
            run += cb[u];
            W.bstart[(kNb / 32) * lane + u + 1] = run;
          }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kOut / 32; ++u) {
          const uint32_t st = lane + 32 * u;
          if (st < n) {
            const uint32_t sp = W.bstart[key[u]] + rank[u];
            W.perm[sp] = (uint8_t)st;
            W.ts[sp] = W.t[st];
          }
        }
        if (lane == 0) {
          W.tmin = tlo;
          W.scale = scale;
          W.m = m;
          W.piece = piece;
        }
        __syncwarp();
        return cnt;
      };

      // incoming cell i of h1: its cell id and inner-layer slot
      auto incoming = [&](uint32_t i, int& kin) -> uint32_t {
        kin = 0;
        while (i >= W.sb[kin + 1]) ++kin;  // i < W.sb[max_inner] bounds the walk
        return W.so[kin] + (i - W.sb[kin]);
      };
      // the first incoming group's inner hits are fetched while the outgoing cells are
      // searched, each later group's while the group before it is processed
      float4 p0_next = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((uint32_t)lane < nin) {
        int kin;
        const uint32_t c0 = incoming(lane, kin);
        if (PT_CHECK(b.cnt, c0 < b.cnt[CNT_CELLS], DBG_CON_INCOMING))
          p0_next = b.hit4[b.cell_in[c0]];
      }
      const uint32_t nout = stage_piece(0);
      if (nout == 0) continue;

      const int npieces = (int)((nout + kOut - 1) / kOut);

      for (uint32_t g0 = 0; g0 < nin; g0 += 32) {
        // the lane's incoming cell
        const uint32_t i = g0 + lane;
        bool valid = i < nin;
        uint32_t c = 0;
        int kin = 0;
        if (valid) {
          c = incoming(i, kin);
          valid = PT_CHECK(b.cnt, c < b.cnt[CNT_CELLS], DBG_CON_INCOMING);
        }
        const float4 p0 = p0_next;
        const bool first_b0 = valid && pt.inner[L1][kin] == 0;
        uint32_t h0_next = 0;
        const bool valid_next = i + 32 < nin;
        if (valid_next) {
          int kn;
          const uint32_t cn = incoming(i + 32, kn);
          if (PT_CHECK(b.cnt, cn < b.cnt[CNT_CELLS], DBG_CON_INCOMING)) h0_next = b.cell_in[cn];
        }
        const float ta = __fdividef(p1.z - p0.z, p1.w - p0.w);  // the cell's slope dz/dr
        const float id1 = __fdividef(1.0f, p1.w - p0.w);
        const float wa = (cuts.rz0 + cuts.rz1 * cuts.cotmax) * id1;
        const float ua = cuts.rz0 + cuts.rz1 * fabsf(ta);
        const float shrink = 1.0f - cuts.rz1 * id1;

        bool inited = false;  // the lane's cell had its out-link list cleared
#pragma unroll 1
        for (int piece = 0; piece < npieces; ++piece) {
          if (W.piece != piece) stage_piece(piece);
          const float m = W.m, tmin = W.tmin, scale = W.scale;
          float w = 0.0f;
          uint32_t pos = 0, pend = 0;
          if (valid) {
            const float im = __fdividef(1.0f, m);
            float wk = fmaf(ua, im, wa);
            if (shrink > 0.0f) wk = fminf(wk, __fdividef(ua * (id1 + im), shrink));
            w = wk * 1.01f + 1e-3f;
            const float w2 = w * 1.001f + 1e-5f;
            pos = W.bstart[slope_bucket(__fsub_rn(ta, w2), tmin, scale)];
            pend = W.bstart[slope_bucket(__fadd_rn(ta, w2), tmin, scale) + 1];
            if (!PT_CHECK(b.cnt, pos <= pend && pend <= (uint32_t)kOut, DBG_CON_BUCKET))
              pend = pos;
          }
          // each lane walks its own bucket range; the staged cells inside its window are
          // queued with their target and tested with C1-C3 once 32 are waiting
          while (__any_sync(kFull, pos < pend)) {
            bool pass = false;
            uint32_t code = 0;
            if (pos < pend) {
              pass = fabsf(W.ts[pos] - ta) <= w;
              if (pass) {
                // the target cell, named by its outer hit and the slot of h1's layer
                // among that hit's inner layers until k_link_targets finds it
                const uint32_t st = W.perm[pos];
                code = W.code[st];
                if (!inited) {
                  b.cell_head[c] = kHole;  // before any of its pairs is tested
                  inited = true;
                }
              }
              ++pos;
            }
            const unsigned bal = __ballot_sync(kFull, pass);
            (void)PT_CHECK(b.cnt, qtail + __popc(bal) - qhead <= (uint32_t)kQueue, DBG_CON_QUEUE);
            if (pass) {
              const uint32_t qi = (qtail + __popc(bal & lt_mask)) & (kQueue - 1);
              W.q[qi] = make_uint4(c, code, h1, first_b0 ? 1u : 0u);
              W.qp0[qi] = p0;
            }
            qtail += __popc(bal);
            if (qtail - qhead >= 32u) process(32u);
          }
        }
        if (valid_next) p0_next = b.hit4[h0_next];
      }
    }
  }
  while (qtail != qhead) process(min(32u, qtail - qhead));
  __syncwarp();
  mark_link_hole(W.chunk_next, W.chunk_end);
  if (lane == 0 && W.used) atomicAdd(&b.cnt[CNT_LINKS_USED], W.used);
}

// Position of inner hit h in the cells [lo, hi) of one segment (ordered by inner hit, each
// inner hit once): the first cell whose inner hit is >= h (hi if none), `found` telling
// whether it is h.  The segment's inner hits spread over the outer hit's window in the
// inner layer, so h's position is guessed from the first and last of them and the eight
// cells around the guess are read at once; a guess that misses leaves a bisection of the
// side beyond it.  Segments of up to eight cells are read whole.  Dependent loads: two or
// three levels for most links, against about seven for a bisection of the whole segment.
__device__ __forceinline__ uint32_t find_inner(const Buffers& b, uint32_t lo, uint32_t hi,
                                               uint32_t h, bool& found) {
  const uint32_t end = hi;
  uint32_t w0 = lo;
  if (hi - lo > 8) {
    const uint32_t f = b.cell_in[lo], la = b.cell_in[hi - 1];
    if (h <= f) {
      found = h == f;
      return lo;
    }
    if (h > la) {
      found = false;
      return hi;
    }
    // f < h <= la
    const uint32_t g =
        lo + (uint32_t)((uint64_t)(h - f) * (uint64_t)(hi - 1 - lo) / (uint64_t)(la - f));
    w0 = min(max(g, lo + 3u) - 3u, hi - 8u);
  }
  // the (up to) eight cells from w0
  uint32_t less = 0;
  bool eq = false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t v = w0 + k < hi ? b.cell_in[w0 + k] : 0xffffffffu;
    less += v < h ? 1u : 0u;
    eq |= v == h;
  }
  if (hi - lo <= 8 || (less > 0 && less < 8)) {
    found = eq;
    return w0 + less;
  }
  // the guess missed: the position lies before w0 (less == 0) or after w0 + 7
  if (less == 0) hi = w0; else lo = w0 + 8;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (b.cell_in[mid] < h) lo = mid + 1; else hi = mid;
  }
  found = lo < end && b.cell_in[lo] == h;
  return lo;
}

// The target cell (h1, h2) of every link: h1 (the outer hit of the source cell) in h2's
// incoming segment from h1's layer, which is ordered by inner hit (find_inner);
// one thread per link slot.  Plain form: the target's incoming-link flag is set and the
// link records the target's out-link list head and outer hit.  Gated
// form: the link's bf16 feature row for the gate's MLP is computed here, one thread per
// link with every lane busy, from the three hits (mostly still in L2).  A
// target can be missing only when the doublet stage ran out of cell slots (its status
// bit is set then); the link then points back to its source, a valid cell, so that the
// later stages stay within their arrays.
template <bool GATE>
__global__ void k_link_targets(Buffers b, pt_cuts cuts, int32_t B, int max_inner,
                               uint64_t cap_links) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = b.link_src[l];
    if (a == kHole) continue;
    const uint32_t t = b.link_dst[l];
    const uint32_t h1 = b.cell_out[a];
    uint2 sg = b.seg[(uint64_t)(t & 0x1fffffffu) * max_inner + (t >> 29)];
    if (!PT_CHECK(b.cnt, (uint64_t)sg.x + sg.y <= b.cnt[CNT_CELLS], DBG_TGT_SEGMENT))
      sg = make_uint2(0u, 0u);
    bool found;
    const uint32_t pos = find_inner(b, sg.x, sg.x + sg.y, h1, found);
    const uint32_t c = found ? pos : a;
    b.link_dst[l] = c;
    if (!GATE) {
      if (found) b.has_in[c] = 1;
      // the target's list (complete: every link was pushed by the link kernel; kHole
      // when the target has none) and outer hit, for the ntuplet walk
      b.link_walk[l] = make_uint2(b.has_out[c] ? b.cell_head[c] : kHole,
                                  found ? (t & 0x1fffffffu) : b.cell_out[c]);
    }
    if (GATE) {
      const uint32_t h0 = b.cell_in[a], h2 = t & 0x1fffffffu;
      float f[kGateFeat];
      gate_link_features(cuts, b.hit4[h0], b.hit4[h1], b.hit4[h2], (b.hbin[h0] / B) % kLayers,
                         (b.hbin[h1] / B) % kLayers, (b.hbin[h2] / B) % kLayers, f);
      store_gate_row(b.gate_x + l * kGateK1, f);
    }
  }
}

}  // namespace

void launch_connect(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                    bool gated) {
  cudaMemsetAsync(&b.cnt[CNT_LNK_WORK], 0, sizeof(unsigned long long), s);  // work counter
  if (gated) {
    PT_TRACE(l, s, "k_connect",
             k_connect<true><<<l.sms * kConnBlocksPerSm, kConnWarps * 32, 0, s>>>(
                 b, p.cuts, p.pairs, p.phi_bins, (uint64_t)p.max_links));
    PT_TRACE(l, s, "k_link_targets",
             k_link_targets<true><<<l.grid, 256, 0, s>>>(b, p.cuts, p.phi_bins, p.pairs.max_inner,
                                                         (uint64_t)p.max_links));
  } else {
    PT_TRACE(l, s, "k_connect",
             k_connect<false><<<l.sms * kConnBlocksPerSm, kConnWarps * 32, 0, s>>>(
                 b, p.cuts, p.pairs, p.phi_bins, (uint64_t)p.max_links));
    PT_TRACE(l, s, "k_link_targets",
             k_link_targets<false><<<l.grid, 256, 0, s>>>(b, p.cuts, p.phi_bins, p.pairs.max_inner,
                                                          (uint64_t)p.max_links));
  }
}

}  // namespace ptca
