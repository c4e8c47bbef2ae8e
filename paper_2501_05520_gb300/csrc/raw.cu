// Raw pixel data -> hits (Sec. 2.2.1 and Fig. 2: the compressed raw data are unpacked
// on the GPU into digis, and neighbouring digis of one layer are clustered into hits).
// The paper fixes no format or algorithm; the library's reading:
//   [P1] a digi is (module, row, col, adc), packed in 64 bits as
//        module << 40 | row << 28 | col << 16 | adc; an event's digis come grouped by
//        module and, within a module, in (row, col) order, each pixel once, adc <= 4095;
//   [P2] a cluster is a set of digis of one module connected through pixels that touch
//        at an edge or a corner;
//   [P3] its hit lies at the adc-weighted mean pixel centre mapped through the module
//        table (barrel: (r cos phi, r sin phi, z); disk: (r cos phi, r sin phi, z_disk));
//   [P4] hits come module run by module run in input order, and within a module in
//        order of their cluster's first pixel.
//
// k_raw_runs flags the start of every module run (a new event or a new module) and
// checks each digi; a scan numbers the runs.  k_raw_cluster gives each run to one warp:
// the run's pixels (already in (row, col) order) go to shared memory with their
// neighbour lists (the pixel to the left and right, and the at most three pixels of the
// rows above and below, found by binary search), each pixel then repeatedly takes the
// smallest label among itself, its label's label and its neighbours until no label
// changes, which leaves every pixel labelled with its cluster's first position; the
// adc-weighted sums are exact integer atomics on those positions, and the positions in
// order give the run's hits at the run's first digi position.  Runs of up to 256 digis
// take one warp each with small buffers (many warps per SM to hide the shared-memory and
// load latency); that launch lists the longer runs (up to 1024), and a second launch
// gives each of those a whole block, which runs the same steps over its pixels.  A
// scan over the runs' hit counts and k_raw_place put the hits of the batch in order into
// the chain's input arrays, with per-event offsets and the batch header.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kRunMax = 1024;           // digis of one module in one event
constexpr int kRunSmall = 256;          // runs of up to this many digis take the small launch
constexpr int kClusterMax = 128;        // pixels of one cluster (32-bit exact sums)
constexpr int kSmallWarps = 4;          // warps per block of the warp-per-run launch (22.5 KB)
constexpr int kSmallBlocksPerSm = 9;
constexpr int kBigThreads = 256;        // block of the block-per-run launch (22.5 KB shared)
constexpr int kBigBlocksPerSm = 4;
constexpr int kLoadBatch = 8;           // digis per lane loaded before use
constexpr uint32_t kAdcMax = 4095;

// Working set of one run of at most CAP pixels (22 bytes a pixel): one per warp in the
// warp-per-run launch, one per block in the block-per-run launch.
template <int CAP>
struct RawWarp {
  uint32_t key[CAP];   // row << 12 | col
  uint32_t nb[CAP];    // neighbour lists (below: first position, count; above: first
                       // position, count; left; right), then the adc sums at the roots
  uint32_t s1[CAP];    // sums at the roots: adc (2 col + 1),
  uint32_t s2[CAP];    //   adc (2 row + 1)
  uint16_t lab[CAP];   // label: a position of the same cluster, finally its first one
  uint16_t adc[CAP];
  uint16_t n[CAP];     // pixels at the roots
};

__device__ __forceinline__ uint32_t digi_module(uint64_t w) { return (uint32_t)(w >> 40); }
__device__ __forceinline__ uint32_t digi_row(uint64_t w) { return (uint32_t)(w >> 28) & 0xfffu; }
__device__ __forceinline__ uint32_t digi_col(uint64_t w) { return (uint32_t)(w >> 16) & 0xfffu; }
__device__ __forceinline__ uint32_t digi_adc(uint64_t w) { return (uint32_t)w & 0xffffu; }

// Event of digi i: largest e with off[e] <= i.
__device__ __forceinline__ int digi_event(const int64_t* off, int E, int64_t i) {
  int lo = 0, hi = E - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// flag[i] = 1 where a module run starts; every digi is checked against the table.
__global__ void k_raw_runs(RawBuffers r, const pt_module* mods, int n_mod, int E,
                           unsigned long long* status) {
  const int64_t n = r.digi_off[E];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.cnt[CNT_RAW_DIGIS] = (unsigned long long)n;
    r.cnt[CNT_RAW_BIG] = 0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = r.words[i];
    const uint32_t m = digi_module(w);
    bool ok = m < (uint32_t)n_mod && digi_adc(w) <= kAdcMax;
    if (ok) ok = digi_row(w) < (uint32_t)mods[m].nrow && digi_col(w) < (uint32_t)mods[m].ncol;
    if (!ok) atomicOr(status, RAW_INVALID);
    const int e = digi_event(r.digi_off, E, i);
    const bool start = i == r.digi_off[e] || digi_module(r.words[i - 1]) != m;
    r.flag[i] = start ? 1u : 0u;
  }
}

// run_first[run] = its first digi (from the scan of the flags); run_first[R] = n.
__global__ void k_raw_run_starts(RawBuffers r, int E) {
  const int64_t n = r.digi_off[E];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (r.flag[i]) r.run_first[r.run_scan[i]] = (uint32_t)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.run_first[r.run_scan[n]] = (uint32_t)n;
    r.cnt[CNT_RAW_RUNS] = r.run_scan[n];
  }
}

// The threads that cluster one run: one warp, or one block.
struct WarpGroup {
  static constexpr uint32_t kSize = 32;
  __device__ uint32_t rank() const { return lane_id(); }
  __device__ void sync() const { __syncwarp(); }
  __device__ bool any(bool p) const {
    const bool q = __any_sync(kFull, p);
    __syncwarp();
    return q;
  }
  __device__ bool all(bool p) const {
    const bool q = __all_sync(kFull, p);
    __syncwarp();
    return q;
  }
  // ranks below this one with p set, and the group's total
  __device__ uint32_t count_below(bool p, uint32_t* total) const {
    const unsigned m = __ballot_sync(kFull, p);
    *total = __popc(m);
    return __popc(m & ((1u << lane_id()) - 1u));
  }
};

template <int THREADS>
struct BlockGroup {
  static constexpr uint32_t kSize = THREADS;
  uint32_t* warp_count;  // shared [THREADS / 32]
  __device__ uint32_t rank() const { return threadIdx.x; }
  __device__ void sync() const { __syncthreads(); }
  __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
  __device__ bool all(bool p) const { return __syncthreads_and(p) != 0; }
  __device__ uint32_t count_below(bool p, uint32_t* total) const {
    const unsigned m = __ballot_sync(kFull, p);
    const uint32_t w = threadIdx.x >> 5;
    if (lane_id() == 0) warp_count[w] = __popc(m);
    __syncthreads();
    uint32_t below = 0, t = 0;
#pragma unroll
    for (int i = 0; i < THREADS / 32; ++i) {
      const uint32_t c = warp_count[i];
      below += (uint32_t)i < w ? c : 0u;
      t += c;
    }
    __syncthreads();
    *total = t;
    return below + __popc(m & ((1u << lane_id()) - 1u));
  }
};

// Clusters of run `run` (digis [s0, s0 + n), n <= CAP) by the group G: the run's pixels
// to shared memory, neighbour lists, labels, sums at the clusters' first positions, one
// hit per cluster in the order of those positions, written at the run's first digi
// position; run_nh[run] = the hits.  Every thread of the group calls it with the same run.
template <int CAP, class G>
__device__ __forceinline__ void cluster_run(const G& g, RawWarp<CAP>& W, const RawBuffers& r,
                                            uint32_t run, uint32_t s0, uint32_t n,
                                            const pt_module* mods, int n_mod,
                                            unsigned long long* status) {
  const uint32_t t = g.rank();
  const uint32_t mi = digi_module(r.words[s0]);
  for (uint32_t k0 = 0; k0 < n; k0 += G::kSize * kLoadBatch) {
    uint64_t wv[kLoadBatch];
#pragma unroll
    for (int i = 0; i < kLoadBatch; ++i) {
      const uint32_t k = k0 + i * G::kSize + t;
      wv[i] = k < n ? r.words[s0 + k] : 0ull;
    }
#pragma unroll
    for (int i = 0; i < kLoadBatch; ++i) {
      const uint32_t k = k0 + i * G::kSize + t;
      if (k < n) {
        W.key[k] = digi_row(wv[i]) << 12 | digi_col(wv[i]);
        W.adc[k] = (uint16_t)digi_adc(wv[i]);
        W.s1[k] = W.s2[k] = 0;
        W.n[k] = 0;
      }
    }
  }
  g.sync();
  bool order_ok = true;
  for (uint32_t k = t + 1; k < n; k += G::kSize) order_ok = order_ok && W.key[k - 1] < W.key[k];
  order_ok = g.all(order_ok);
  if (mi >= (uint32_t)n_mod || !order_ok) {  // a bad module is flagged by k_raw_runs
    if (t == 0) {
      if (mi < (uint32_t)n_mod) atomicOr(status, RAW_INVALID);
      r.run_nh[run] = 0;
    }
    return;
  }
  const pt_module md = mods[mi];
  // neighbour lists: in (row, col) order the pixels of the rows above and below within
  // one column of this one are contiguous, at most three each; the first label is the
  // smallest neighbour position (above, else left, else the pixel itself)
  for (uint32_t k = t; k < n; k += G::kSize) {
    const uint32_t key = W.key[k], row = key >> 12, col = key & 0xfffu;
    const uint32_t c0 = col > 0 ? col - 1u : 0u, c1 = col < 0xfffu ? col + 1u : col;
    uint32_t lo = k + 1, hi = n;
    const uint32_t wl = (row + 1u) << 12 | c0;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (W.key[mid] < wl) lo = mid + 1; else hi = mid;
    }
    uint32_t lc = 0;
    while (lc < 3 && lo + lc < n && W.key[lo + lc] <= ((row + 1u) << 12 | c1)) ++lc;
    uint32_t uo = 0, uc = 0;
    if (row > 0) {
      uint32_t a = 0, z = k;
      const uint32_t wu = (row - 1u) << 12 | c0;
      while (a < z) {
        const uint32_t mid = (a + z) >> 1;
        if (W.key[mid] < wu) a = mid + 1; else z = mid;
      }
      uo = a;
      while (uc < 3 && uo + uc < k && W.key[uo + uc] <= ((row - 1u) << 12 | c1)) ++uc;
    }
    const bool left = col > 0 && k > 0 && W.key[k - 1] == key - 1u;
    const bool right = col < 0xfffu && k + 1 < n && W.key[k + 1] == key + 1u;
    W.nb[k] = lo | lc << 11 | uo << 13 | uc << 24 | (left ? 1u << 26 : 0u) |
              (right ? 1u << 27 : 0u);
    W.lab[k] = (uint16_t)(uc ? uo : left ? k - 1 : k);
  }
  g.sync();
  // every pixel takes the smallest of its label, its label's label and its neighbours'
  // labels; labels only fall and stay positions of the pixel's cluster, and once none
  // changes each equals its cluster's smallest position (at most one pass per pixel of
  // the longest path, and one more to see that nothing changed)
  volatile uint16_t* lab = W.lab;
  bool changed = true;
  for (int pass = 0; pass <= CAP && changed; ++pass) {
    changed = false;
    for (uint32_t k = t; k < n; k += G::kSize) {
      const uint32_t nb = W.nb[k];
      const uint32_t cur = lab[k];
      uint32_t m = min(cur, (uint32_t)lab[cur]);
      if (nb & (1u << 26)) m = min(m, (uint32_t)lab[k - 1]);
      if (nb & (1u << 27)) m = min(m, (uint32_t)lab[k + 1]);
      const uint32_t lo = nb & 0x7ffu, lc = (nb >> 11) & 3u;
      const uint32_t uo = (nb >> 13) & 0x7ffu, uc = (nb >> 24) & 3u;
      for (uint32_t i = 0; i < lc; ++i) m = min(m, (uint32_t)lab[lo + i]);
      for (uint32_t i = 0; i < uc; ++i) m = min(m, (uint32_t)lab[uo + i]);
      if (m < cur) {
        lab[k] = (uint16_t)m;
        changed = true;
      }
    }
    changed = g.any(changed);
  }
  if (changed && t == 0) atomicOr(status, RAW_INVALID);
  for (uint32_t k = t; k < n; k += G::kSize) W.nb[k] = 0;
  g.sync();
  // sums at the roots (exact: adc <= 4095, 2 col + 1 < 8192, <= 128 pixels)
  for (uint32_t k = t; k < n; k += G::kSize) {
    const uint32_t root = W.lab[k];
    const uint32_t adc = W.adc[k];
    const uint32_t row = W.key[k] >> 12, col = W.key[k] & 0xfffu;
    atomicAdd(&W.nb[root], adc);
    atomicAdd(&W.s1[root], adc * (2u * col + 1u));
    atomicAdd(&W.s2[root], adc * (2u * row + 1u));
    atomicAdd(reinterpret_cast<unsigned int*>(&W.n[root & ~1u]), 1u << ((root & 1u) * 16u));
  }
  g.sync();
  // roots in order -> hits
  uint32_t nh = 0;
  for (uint32_t k0 = 0; k0 < n; k0 += G::kSize) {
    const uint32_t k = k0 + t;
    const bool root = k < n && W.lab[k] == k;
    uint32_t total;
    const uint32_t below = g.count_below(root, &total);
    if (root) {
      if (W.n[k] > (uint16_t)kClusterMax) atomicOr(status, RAW_CLUSTER_CAPACITY);
      const float w2 = 2.0f * (float)W.nb[k];
      const float col_c = (float)W.s1[k] / w2, row_c = (float)W.s2[k] / w2;
      const float phi = md.phi0 + col_c * md.dphi_col;
      const float v = md.v0 + row_c * md.dv_row;
      float sn, cs;
      sincosf(phi, &sn, &cs);
      const float rad = md.kind == 0 ? md.rz : v;
      r.stage[s0 + nh + below] = make_float4(rad * cs, rad * sn, md.kind == 0 ? v : md.rz,
                                             __int_as_float(md.layer));
    }
    nh += total;
  }
  if (t == 0) r.run_nh[run] = nh;
  g.sync();
}

// One warp per run of at most kRunSmall digis; longer runs go to the block-per-run
// launch's list.
__global__ void __launch_bounds__(kSmallWarps * 32, kSmallBlocksPerSm)
    k_raw_cluster(RawBuffers r, const pt_module* mods, int n_mod, unsigned long long* status) {
  __shared__ RawWarp<kRunSmall> s_w[kSmallWarps];
  RawWarp<kRunSmall>& W = s_w[threadIdx.x >> 5];
  const uint32_t R = r.run_scan[r.digi_off[r.n_events]];
  const uint32_t nwarps = gridDim.x * kSmallWarps;
  uint32_t run = blockIdx.x * kSmallWarps + (threadIdx.x >> 5);
  uint32_t s = 0, e = 0;
  if (run < R) {
    s = r.run_first[run];
    e = r.run_first[run + 1];
  }
  for (; run < R; run += nwarps) {
    // the next run's bounds, loaded while this one is clustered
    const uint32_t nrun = run + nwarps;
    uint32_t ns = 0, ne = 0;
    if (nrun < R) {
      ns = r.run_first[nrun];
      ne = r.run_first[nrun + 1];
    }
    const uint32_t s0 = s, n = e - s;
    s = ns;
    e = ne;
    if (n > (uint32_t)kRunSmall) {
      if (lane_id() == 0) r.big_runs[atomicAdd(&r.cnt[CNT_RAW_BIG], 1ull)] = run;
      continue;
    }
    cluster_run<kRunSmall>(WarpGroup{}, W, r, run, s0, n, mods, n_mod, status);
  }
}

// One block per listed run of more than kRunSmall digis (at most kRunMax).
__global__ void __launch_bounds__(kBigThreads, kBigBlocksPerSm)
    k_raw_cluster_big(RawBuffers r, const pt_module* mods, int n_mod, unsigned long long* status) {
  __shared__ RawWarp<kRunMax> W;
  __shared__ uint32_t s_count[kBigThreads / 32];
  const BlockGroup<kBigThreads> g{s_count};
  const uint32_t nbig = (uint32_t)r.cnt[CNT_RAW_BIG];
  for (uint32_t i = blockIdx.x; i < nbig; i += gridDim.x) {
    const uint32_t run = r.big_runs[i];
    const uint32_t s0 = r.run_first[run], n = r.run_first[run + 1] - s0;
    if (n > (uint32_t)kRunMax) {
      if (threadIdx.x == 0) {
        atomicOr(status, RAW_RUN_CAPACITY);
        r.run_nh[run] = 0;
      }
      continue;
    }
    cluster_run<kRunMax>(g, W, r, run, s0, n, mods, n_mod, status);
  }
}

// Hits of run `run` to the chain's inputs at run_hoff[run]; per-event hit offsets (an
// event's first run; events without digis own no hits) and the batch header.
__global__ void k_raw_place(RawBuffers r, Buffers b, int64_t cap_hits, unsigned long long* status) {
  const int E = r.n_events;
  const uint32_t R = r.run_scan[r.digi_off[E]];
  const uint32_t H = r.run_hoff[R];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    if ((int64_t)H > cap_hits) atomicOr(status, RAW_HIT_CAPACITY);
    b.hdr->n_events = E;
    b.hdr->n_hits = (int32_t)min((int64_t)H, cap_hits);
    r.cnt[CNT_RAW_HITS] = H;
  }
  for (int64_t e = tid; e <= E; e += stride) {
    // first run whose first digi is at or after the event's first digi
    const int64_t d = r.digi_off[e];
    uint32_t lo = 0, hi = R;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((int64_t)r.run_first[mid] < d) lo = mid + 1; else hi = mid;
    }
    b.hit_off[e] = (int32_t)min((int64_t)r.run_hoff[lo], cap_hits);
  }
  // one warp per run, one lane per hit
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nw = (uint32_t)(stride >> 5);
  for (uint32_t run = (uint32_t)(tid >> 5); run < R; run += nw) {
    const uint32_t s = r.run_first[run], h0 = r.run_hoff[run], nh = r.run_nh[run];
    for (uint32_t k = lane; k < nh; k += 32) {
      if ((int64_t)(h0 + k) >= cap_hits) break;
      const float4 p = r.stage[s + k];
      b.in_x[h0 + k] = p.x;
      b.in_y[h0 + k] = p.y;
      b.in_z[h0 + k] = p.z;
      b.in_layer[h0 + k] = (uint8_t)__float_as_int(p.w);
    }
  }
}

}  // namespace

cudaError_t launch_raw(const RawBuffers& r, const Buffers& b, const pt_module* mods, int n_mod,
                       int64_t cap_hits, const Launch& l, cudaStream_t s) {
  unsigned long long* status = &b.cnt[CNT_RAW_STATUS];
  PT_TRACE(l, s, "k_raw_runs", k_raw_runs<<<l.grid, 256, 0, s>>>(r, mods, n_mod, r.n_events, status));
  // run numbers: run_scan[i] = runs starting before digi i
  PT_TRACE(l, s, "scan", launch_scan(r.flag, r.run_scan, &r.cnt[CNT_RAW_DIGIS], r.scan_part, s));
  PT_TRACE(l, s, "k_raw_run_starts", k_raw_run_starts<<<l.grid, 256, 0, s>>>(r, r.n_events));
  PT_TRACE(l, s, "k_raw_cluster",
           k_raw_cluster<<<l.sms * kSmallBlocksPerSm, kSmallWarps * 32, 0, s>>>(r, mods, n_mod,
                                                                                status));
  PT_TRACE(l, s, "k_raw_cluster_big",
           k_raw_cluster_big<<<l.sms * kBigBlocksPerSm, kBigThreads, 0, s>>>(r, mods, n_mod,
                                                                             status));
  PT_TRACE(l, s, "scan", launch_scan(r.run_nh, r.run_hoff, &r.cnt[CNT_RAW_RUNS], r.scan_part, s));
  PT_TRACE(l, s, "k_raw_place", k_raw_place<<<l.grid, 256, 0, s>>>(r, b, cap_hits, status));
  return cudaGetLastError();
}

}  // namespace ptca
