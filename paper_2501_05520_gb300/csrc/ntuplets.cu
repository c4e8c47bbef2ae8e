// Stages A4-A6: ntuplet extraction, canonical order and duplicate cleaning (Sec.
// 2.2.1, Fig. 2: starting from the seeds, the chain selects the sets of hits that are
// candidate tracks).
//
// A4  every path of linked cells from a root (a cell with no incoming link) to a leaf
//     (a cell with no outgoing link) with 3..6 hits.  Roots are taken among the sources
//     of the link lists (a root without an outgoing link would give a 2-hit path,
//     which is dropped).  One thread per root walks its out-links depth first with an
//     explicit stack (the layer graph bounds the depth at 5 cells), writing the paths to
//     its warp's shared buffer, which one atomic per 32 roots reserves and the warp
//     copies out (a batch of roots with more paths than the buffer holds is walked a
//     second time and written directly).  The path quality q is the float32 sum of its link qualities,
//     added from the innermost link outwards.
// A6  canonical order: ntuplets sorted by their hit tuple (batch input indices, -1
//     padded, signed).  A counting sort on the first hit puts them in per-hit buckets
//     (a few entries each), which one thread per bucket finishes by insertion sort.
// A5  duplicate cleaning on the sorted list, rank i = sorted position: key =
//     (6 - nhits, q bits, i) packed in 64 bits, so a smaller key is "more hits, then
//     smaller q, then smaller tuple".  atomicMin gives every cell its best key; an
//     ntuplet survives when it holds the best key of all its cells; a triplet then
//     dies if it shares a hit with a surviving ntuplet of >= 4 hits.  Survivors are
//     compacted in sorted order, and per-event offsets are derived from it.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

// Ntuplets buffered per warp in shared memory before one global reservation, and the
// search's blocks per SM (more walks in flight hide more of their load latency; the
// build may set both for tuning sweeps).
#ifndef PT_NT_BUF
#define PT_NT_BUF 64
#endif
#ifndef PT_NT_BLOCKS_PER_SM
#define PT_NT_BLOCKS_PER_SM 6
#endif
constexpr int kNtBuf = PT_NT_BUF;
constexpr int kNtWarps = 8;  // warps per block of the ntuplet search
constexpr int kNtBlocksPerSm = PT_NT_BLOCKS_PER_SM;
struct NtWarp {
  uint32_t roots[64];                        // queued roots (< 32 + 32)
  int32_t hits[kNtBuf][kMaxHits];            // buffered ntuplets (sorted hit indices)
  uint32_t cells[kNtBuf][kMaxCellsPerNt];
  float q[kNtBuf];
  uint32_t n[kNtBuf];
  uint32_t cnt;                              // ntuplets found by the batch (may exceed kNtBuf)
};

enum WalkMode { kCount = 0, kEmit = 1, kBuffer = 2 };

// Depth-first walk from root a.  kCount: returns the number of ntuplets; kEmit: also
// writes them at slots t0, t0 + 1, ... (slots >= cap_nt are dropped); kBuffer: also
// writes them to the warp's shared buffer (entries >= kNtBuf are dropped; the caller
// then walks again with kEmit).  A cell's links are a list (its head, then each link's
// next slot).  The walk keeps the sorted index of each cell's outer hit, read beside
// the cell's flag and list head when the cell is pushed, so that no step waits on a
// third dependent load; the batch index (perm) is looked up when a path is written
// (kEmit) or when the warp copies its buffer out (kBuffer holds sorted indices).
template <int MODE, bool GATED>
__device__ uint32_t walk(const Buffers& b, uint32_t a, unsigned long long t0, uint64_t cap_nt,
                         NtWarp* W) {
  constexpr bool EMIT = MODE != kCount;
  uint32_t path[kMaxCellsPerNt];
  uint32_t it[kMaxCellsPerNt];  // next out-link slot of path[k] (kHole: none left)
  float qs[kMaxCellsPerNt];
  int32_t gh[kMaxCellsPerNt];  // sorted index of the outer hit of path[k] (EMIT)
  // a link slot read from the lists (debug build: kHole unless inside the link slots)
  auto slot = [&](uint32_t x) -> uint32_t {
    return (x == kHole || PT_CHECK(b.cnt, x < b.cnt[CNT_LINKS], DBG_NT_LINKS)) ? x : kHole;
  };
  path[0] = a;
  it[0] = slot(b.cell_head[a]);
  qs[0] = 0.0f;
  int32_t g0 = 0;
  if (EMIT) {
    g0 = (int32_t)b.cell_in[a];
    gh[0] = (int32_t)b.cell_out[a];
  }
  uint32_t found = 0;
  int depth = 1;
  while (depth > 0) {
    const int d = depth - 1;
    if (it[d] == kHole) {
      --depth;
      continue;
    }
    const uint32_t l = it[d];
    it[d] = slot(b.link_next[l]);
    if (depth == kMaxCellsPerNt) continue;  // deeper than the layer graph allows
    if (GATED && !b.gate_keep[l]) continue;  // removed by the learned gate
    const uint32_t c = b.link_dst[l];
    if (!PT_CHECK(b.cnt, c < b.cnt[CNT_CELLS], DBG_NT_CELL)) continue;
    const float q = fadd(qs[d], b.link_q[l]);
    bool leaf;
    uint32_t hc;
    int32_t gc;
    if (!GATED) {
      // the link carries c's list head (kHole: c is a leaf) and outer hit, so a step
      // waits on one level of loads
      const uint2 w = b.link_walk[l];
      leaf = w.x == kHole;
      hc = w.x;
      gc = (int32_t)w.y;
    } else {
      // everything c may need is loaded at once: its flag, its list head (stale and
      // unused when c has no links; it also holds the links the mask removed) and its
      // outer hit
      leaf = !b.has_out[c];
      hc = b.cell_head[c];
      gc = EMIT ? (int32_t)b.cell_out[c] : 0;
    }
    if (leaf) {
      // leaf: path[0..d] + c, i.e. depth + 1 cells, depth + 2 hits
      if (EMIT) {
        const int ncell = depth + 1;
        const int32_t gl = gc;
        int32_t* hp = nullptr;
        uint32_t* cp = nullptr;
        bool keep = false;
        if (MODE == kEmit) {
          const unsigned long long t = t0 + found;
          keep = t < cap_nt;
          if (keep) {
            hp = b.nt_hits + t * kMaxHits;
            cp = b.nt_cells + t * kMaxCellsPerNt;
            b.nt_n[t] = (uint8_t)(ncell + 1);
            b.nt_q[t] = q;
          }
        } else {
          const uint32_t e = atomicAdd(&W->cnt, 1u);
          keep = e < (uint32_t)kNtBuf;
          if (keep) {
            hp = W->hits[e];
            cp = W->cells[e];
            W->n[e] = (uint32_t)(ncell + 1);
            W->q[e] = q;
          }
        }
        for (int k = 0; k < ncell; ++k)
          b.best[k < depth ? path[k] : c] = ~0ull;  // initial duplicate-cleaning key
        if (keep) {
          // batch indices when written out, sorted ones in the warp's buffer
          auto hit = [&](int32_t sorted) -> int32_t {
            return MODE == kEmit ? (int32_t)b.perm[sorted] : sorted;
          };
          hp[0] = hit(g0);
          for (int k = 0; k < ncell; ++k) {
            hp[k + 1] = hit(k < depth ? gh[k] : gl);
            cp[k] = k < depth ? path[k] : c;
          }
          for (int k = ncell + 1; k < kMaxHits; ++k) hp[k] = -1;
          for (int k = ncell; k < kMaxCellsPerNt; ++k) cp[k] = 0xffffffffu;
        }
      }
      ++found;
      continue;
    }
    path[depth] = c;
    it[depth] = slot(hc);
    qs[depth] = q;
    if (EMIT) gh[depth] = gc;
    ++depth;
  }
  return found;
}

// The slot that heads a source cell's out-link list names a candidate root, which is a
// root when the cell has a kept outgoing link and no incoming one.  Each warp queues the roots of its link slots in
// shared memory and walks them 32 at a time, one per lane, writing the ntuplets to its
// shared buffer; one atomic then reserves them and the warp copies them out.  If a
// batch finds more than the buffer holds, it is walked again and written directly.
template <bool GATED>
__global__ void __launch_bounds__(kNtWarps * 32, kNtBlocksPerSm)
    k_find_ntuplets(Buffers b, uint64_t cap_links, uint64_t cap_nt) {
  __shared__ NtWarp s_w[kNtWarps];
  NtWarp& W = s_w[threadIdx.x >> 5];
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const int lane = lane_id();
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t nq = 0;  // queued roots (warp-uniform)
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < nl;
       i0 += stride) {
    const uint64_t i = i0 + lane;
    uint32_t a = kHole;
    if (i < nl) a = b.link_src[i];
    const bool root = a != kHole && b.cell_head[a] == (uint32_t)i && b.has_out[a] && !b.has_in[a];
    const unsigned rm = __ballot_sync(kFull, root);
    if (root) W.roots[nq + __popc(rm & lt_mask)] = a;
    nq += __popc(rm);
    const bool final = i0 + stride >= nl;
    while (nq >= 32u || (final && nq > 0u)) {
      const uint32_t take = min(nq, 32u);
      __syncwarp();
      const uint32_t r = (uint32_t)lane < take ? W.roots[lane] : kHole;
      if (lane == 0) W.cnt = 0;
      __syncwarp();
      const uint32_t n = r != kHole ? walk<kBuffer, GATED>(b, r, 0, cap_nt, &W) : 0u;
      __syncwarp();
      const uint32_t tot = W.cnt;
      // the roots not taken move to the front of the queue
      const uint32_t rest = nq - take;
      const uint32_t moved = (uint32_t)lane < rest ? W.roots[take + lane] : 0u;
      __syncwarp();
      if ((uint32_t)lane < rest) W.roots[lane] = moved;
      nq = rest;
      if (tot == 0) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&b.cnt[CNT_NT], (unsigned long long)tot);
      base = __shfl_sync(kFull, base, 0);
      if (base + tot > cap_nt && lane == 0) atomicOr(&b.cnt[CNT_STATUS], ST_NT);
      if (tot <= (uint32_t)kNtBuf) {
        for (uint32_t e = lane; e < tot; e += 32) {
          const unsigned long long t = base + e;
          if (t < cap_nt) {
#pragma unroll
            for (int k = 0; k < kMaxHits; ++k) {
              const int32_t sh = W.hits[e][k];  // sorted index, -1 pad
              b.nt_hits[t * kMaxHits + k] = sh >= 0 ? (int32_t)b.perm[sh] : -1;
            }
#pragma unroll
            for (int k = 0; k < kMaxCellsPerNt; ++k)
              b.nt_cells[t * kMaxCellsPerNt + k] = W.cells[e][k];
            b.nt_n[t] = (uint8_t)W.n[e];
            b.nt_q[t] = W.q[e];
          }
        }
      } else {
        const uint32_t inc = warp_incl_scan(n);
        if (n) walk<kEmit, GATED>(b, r, base + inc - n, cap_nt, &W);
      }
    }
  }
}

__global__ void k_bucket_count(Buffers b, uint64_t cap_nt) {
  const uint64_t T = min(b.cnt[CNT_NT], (unsigned long long)cap_nt);
  if (blockIdx.x == 0 && threadIdx.x == 0) b.cnt[CNT_SCAN_NT] = T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride)
    b.nt_rank[t] = atomicAdd(&b.bucket_cnt[b.nt_hits[t * kMaxHits]], 1u);
}

__global__ void k_bucket_scatter(Buffers b, uint64_t cap_nt) {
  const uint64_t T = min(b.cnt[CNT_NT], (unsigned long long)cap_nt);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride)
    b.ord[b.bucket_start[b.nt_hits[t * kMaxHits]] + b.nt_rank[t]] = (uint32_t)t;
}

__device__ __forceinline__ bool tuple_less(const int32_t* a, const int32_t* c) {
#pragma unroll
  for (int k = 1; k < kMaxHits; ++k) {
    if (a[k] != c[k]) return a[k] < c[k];
  }
  return false;
}

__global__ void k_bucket_sort(Buffers b) {
  const int N = b.hdr->n_hits;
  const int stride = gridDim.x * blockDim.x;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < N; h += stride) {
    const uint32_t lo = b.bucket_start[h], hi = b.bucket_start[h + 1];
    for (uint32_t i = lo + 1; i < hi; ++i) {
      const uint32_t v = b.ord[i];
      const int32_t* hv = b.nt_hits + (uint64_t)v * kMaxHits;
      uint32_t j = i;
      while (j > lo && tuple_less(hv, b.nt_hits + (uint64_t)b.ord[j - 1] * kMaxHits)) {
        b.ord[j] = b.ord[j - 1];
        --j;
      }
      b.ord[j] = v;
    }
    for (uint32_t i = lo; i < hi; ++i) b.nt_rank[b.ord[i]] = i;  // sorted position
  }
}

__device__ __forceinline__ unsigned long long dedup_key(const Buffers& b, uint32_t t, uint64_t i) {
  return ((unsigned long long)(kMaxHits - b.nt_n[t]) << 61) |
         ((unsigned long long)__float_as_uint(b.nt_q[t]) << kRankBits) | i;
}

// The two key kernels take the candidates in their own order (their arrays read
// contiguously) and find each one's sorted position in nt_rank.
__global__ void k_dedup_min(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride) {
    const uint32_t i = b.nt_rank[t];
    const unsigned long long key = dedup_key(b, (uint32_t)t, i);
    const int nc = b.nt_n[t] - 1;
    for (int k = 0; k < nc; ++k) atomicMin(&b.best[b.nt_cells[(uint64_t)t * kMaxCellsPerNt + k]], key);
  }
}

__global__ void k_dedup_alive(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride) {
    const uint32_t i = b.nt_rank[t];
    const unsigned long long key = dedup_key(b, (uint32_t)t, i);
    const int n = b.nt_n[t];
    bool ok = true;
    for (int k = 0; k < n - 1; ++k)
      ok = ok && (b.best[b.nt_cells[(uint64_t)t * kMaxCellsPerNt + k]] == key);
    b.alive[i] = ok ? 1u : 0u;
    if (ok && n >= 4)
      for (int k = 0; k < n; ++k) b.used[b.nt_hits[(uint64_t)t * kMaxHits + k]] = 1;
  }
}

__global__ void k_dedup_triplets(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    if (!b.alive[i]) continue;
    const uint32_t t = b.ord[i];
    if (b.nt_n[t] != 3) continue;
    const int32_t* h = b.nt_hits + (uint64_t)t * kMaxHits;
    if (b.used[h[0]] || b.used[h[1]] || b.used[h[2]]) b.alive[i] = 0u;
  }
}

__global__ void k_compact(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) b.cnt[CNT_SV] = b.alive_scan[T];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride)
    if (b.alive[i]) b.sv[b.alive_scan[i]] = (uint32_t)i;
}

// ev_nt_off[e] = first survivor of event >= e; survivors are ordered by event because
// batch input indices are.
__global__ void k_event_offsets(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const uint64_t S = b.alive_scan[T];
  const int E = b.hdr->n_events;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= S; j += stride) {
    const int e_cur = j < S ? find_event(b.hit_off, E, b.nt_hits[(uint64_t)b.ord[b.sv[j]] * kMaxHits])
                            : E;
    const int e_prev =
        j > 0 ? find_event(b.hit_off, E, b.nt_hits[(uint64_t)b.ord[b.sv[j - 1]] * kMaxHits]) : -1;
    for (int e = e_prev + 1; e <= e_cur; ++e) b.ev_nt_off[e] = (int64_t)j;
  }
}

}  // namespace

void launch_ntuplets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                     bool gated) {
  const uint64_t cap_nt = (uint64_t)p.max_ntuplets;
  if (gated)
    PT_TRACE(l, s, "k_find_ntuplets",
             k_find_ntuplets<true><<<l.sms * kNtBlocksPerSm, kNtWarps * 32, 0, s>>>(
                 b, (uint64_t)p.max_links, cap_nt));
  else
    PT_TRACE(l, s, "k_find_ntuplets",
             k_find_ntuplets<false><<<l.sms * kNtBlocksPerSm, kNtWarps * 32, 0, s>>>(
                 b, (uint64_t)p.max_links, cap_nt));
  PT_TRACE(l, s, "k_bucket_count", k_bucket_count<<<l.grid, 256, 0, s>>>(b, cap_nt));
  PT_TRACE(l, s, "scan",
           launch_scan(b.bucket_cnt, b.bucket_start, &b.cnt[CNT_SCAN_HITS], b.scan_part, s));
  PT_TRACE(l, s, "k_bucket_scatter", k_bucket_scatter<<<l.grid, 256, 0, s>>>(b, cap_nt));
  PT_TRACE(l, s, "k_bucket_sort", k_bucket_sort<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "k_dedup_min", k_dedup_min<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "k_dedup_alive", k_dedup_alive<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "k_dedup_triplets", k_dedup_triplets<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "scan", launch_scan(b.alive, b.alive_scan, &b.cnt[CNT_SCAN_NT], b.scan_part, s));
  PT_TRACE(l, s, "k_compact", k_compact<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "k_event_offsets", k_event_offsets<<<l.grid, 256, 0, s>>>(b));
}

}  // namespace ptca
