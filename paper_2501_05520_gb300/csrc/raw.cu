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
// the run's pixels (at most 1024, already in (row, col) order) go to shared memory,
// each pixel joins its right-hand and three lower neighbours (found by binary search)
// in a union-find whose roots are the smallest member positions, the adc-weighted sums
// are exact integer atomics on the roots, and the roots in order give the run's hits at
// the run's first digi position.  A scan over the runs' hit counts and k_raw_place put
// the hits of the batch in order into the chain's input arrays, with per-event offsets
// and the batch header.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kRunMax = 1024;           // digis of one module in one event
constexpr int kClusterMax = 128;        // pixels of one cluster (32-bit exact sums)
constexpr int kRawWarps = 2;            // warps per block of k_raw_cluster (40 KB shared)
constexpr int kRawBlocksPerSm = 5;
constexpr uint32_t kAdcMax = 4095;

struct RawWarp {
  uint32_t key[kRunMax];      // row << 12 | col
  uint16_t parent[kRunMax];   // union-find (root = smallest member position)
  uint32_t s0[kRunMax];       // sums at the roots: adc,
  uint32_t s1[kRunMax];       //   adc (2 col + 1),
  uint32_t s2[kRunMax];       //   adc (2 row + 1),
  uint16_t n[kRunMax];        //   pixels
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
  if (blockIdx.x == 0 && threadIdx.x == 0) r.cnt[CNT_RAW_DIGIS] = (unsigned long long)n;
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

__device__ __forceinline__ uint32_t uf_find(volatile uint16_t* parent, uint32_t x) {
  for (int it = 0; it < kRunMax && parent[x] != x; ++it) x = parent[x];
  return x;
}

// Joins the sets of a and b: the larger root is hooked under the smaller with a
// compare-and-swap, retried from the new roots if another lane moved it first.
__device__ __forceinline__ bool uf_unite(uint16_t* parent, uint32_t a, uint32_t b) {
  volatile uint16_t* vp = parent;
  for (int it = 0; it < 4 * kRunMax; ++it) {
    a = uf_find(vp, a);
    b = uf_find(vp, b);
    if (a == b) return true;
    if (a > b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    // 16-bit CAS through the containing 32-bit word
    uint32_t* word = reinterpret_cast<uint32_t*>(parent + (b & ~1u));
    const uint32_t sh = (b & 1u) * 16u;
    const uint32_t cur = *reinterpret_cast<volatile uint32_t*>(word);
    if (((cur >> sh) & 0xffffu) != b) continue;  // b is no longer a root
    const uint32_t want = (cur & ~(0xffffu << sh)) | (a << sh);
    if (atomicCAS(word, cur, want) == cur) return true;
  }
  return false;
}

// One warp per module run: union-find of its pixels, sums at the roots, one hit per
// root written at the run's first digi position.
__global__ void __launch_bounds__(kRawWarps * 32) k_raw_cluster(RawBuffers r, const pt_module* mods,
                                                                int n_mod,
                                                                unsigned long long* status) {
  __shared__ RawWarp s_w[kRawWarps];
  RawWarp& W = s_w[threadIdx.x >> 5];
  const int lane = lane_id();
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t R = r.run_scan[r.digi_off[r.n_events]];
  const uint32_t nwarps = gridDim.x * kRawWarps;
  for (uint32_t run = blockIdx.x * kRawWarps + (threadIdx.x >> 5); run < R; run += nwarps) {
    const uint32_t s = r.run_first[run], n = r.run_first[run + 1] - s;
    if (n > (uint32_t)kRunMax) {
      if (lane == 0) {
        atomicOr(status, RAW_RUN_CAPACITY);
        r.run_nh[run] = 0;
      }
      continue;
    }
    const uint32_t mi = digi_module(r.words[s]);
    if (mi >= (uint32_t)n_mod) {  // flagged by k_raw_runs
      if (lane == 0) r.run_nh[run] = 0;
      continue;
    }
    const pt_module md = mods[mi];
    bool order_ok = true;
    for (uint32_t k = lane; k < n; k += 32) {
      const uint64_t w = r.words[s + k];
      const uint32_t key = digi_row(w) << 12 | digi_col(w);
      W.key[k] = key;
      W.parent[k] = (uint16_t)k;
      W.s0[k] = W.s1[k] = W.s2[k] = 0;
      W.n[k] = 0;
      if (k > 0) {
        const uint64_t wp = r.words[s + k - 1];
        order_ok = order_ok && (digi_row(wp) << 12 | digi_col(wp)) < key;
      }
    }
    if (!__all_sync(kFull, order_ok)) {
      if (lane == 0) {
        atomicOr(status, RAW_INVALID);
        r.run_nh[run] = 0;
      }
      continue;
    }
    __syncwarp();
    bool joined = true;
    for (uint32_t k = lane; k < n; k += 32) {
      const uint32_t row = W.key[k] >> 12, col = W.key[k] & 0xfffu;
      if (col < 0xfffu && k + 1 < n && W.key[k + 1] == W.key[k] + 1u)
        joined &= uf_unite(W.parent, k, k + 1);
      // first pixel of the next row at or after col - 1
      const uint32_t want = (row + 1u) << 12 | (col > 0 ? col - 1u : 0u);
      uint32_t lo = k + 1, hi = n;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (W.key[mid] < want) lo = mid + 1; else hi = mid;
      }
      const uint32_t last = (row + 1u) << 12 | (col < 0xfffu ? col + 1u : col);
      for (uint32_t j = lo; j < n && W.key[j] <= last; ++j)
        joined &= uf_unite(W.parent, k, j);
    }
    if (!__all_sync(kFull, joined) && lane == 0) atomicOr(status, RAW_INVALID);
    __syncwarp();
    // sums at the roots (exact: adc <= 4095, 2 col + 1 < 8192, <= 128 pixels)
    for (uint32_t k = lane; k < n; k += 32) {
      const uint32_t root = uf_find(W.parent, k);
      const uint32_t adc = digi_adc(r.words[s + k]);
      const uint32_t row = W.key[k] >> 12, col = W.key[k] & 0xfffu;
      atomicAdd(&W.s0[root], adc);
      atomicAdd(&W.s1[root], adc * (2u * col + 1u));
      atomicAdd(&W.s2[root], adc * (2u * row + 1u));
      atomicAdd(reinterpret_cast<unsigned int*>(&W.n[root & ~1u]), 1u << ((root & 1u) * 16u));
    }
    __syncwarp();
    // roots in order -> hits
    uint32_t nh = 0;
    for (uint32_t k0 = 0; k0 < n; k0 += 32) {
      const uint32_t k = k0 + lane;
      const bool root = k < n && W.parent[k] == k;
      const unsigned rm = __ballot_sync(kFull, root);
      if (root) {
        const uint32_t h = s + nh + __popc(rm & lt_mask);
        if (W.n[k] > (uint16_t)kClusterMax) atomicOr(status, RAW_CLUSTER_CAPACITY);
        const float w2 = 2.0f * (float)W.s0[k];
        const float col_c = (float)W.s1[k] / w2, row_c = (float)W.s2[k] / w2;
        const float phi = md.phi0 + col_c * md.dphi_col;
        const float v = md.v0 + row_c * md.dv_row;
        float sn, cs;
        sincosf(phi, &sn, &cs);
        const float rad = md.kind == 0 ? md.rz : v;
        r.stage[h] = make_float4(rad * cs, rad * sn, md.kind == 0 ? v : md.rz,
                                 __int_as_float(md.layer));
      }
      nh += __popc(rm);
    }
    if (lane == 0) r.run_nh[run] = nh;
    __syncwarp();
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
  for (uint32_t run = (uint32_t)tid; run < R; run += (uint32_t)stride) {
    const uint32_t s = r.run_first[run], h0 = r.run_hoff[run], nh = r.run_nh[run];
    for (uint32_t k = 0; k < nh; ++k) {
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
           k_raw_cluster<<<l.sms * kRawBlocksPerSm, kRawWarps * 32, 0, s>>>(r, mods, n_mod,
                                                                             status));
  PT_TRACE(l, s, "scan", launch_scan(r.run_nh, r.run_hoff, &r.cnt[CNT_RAW_RUNS], r.scan_part, s));
  PT_TRACE(l, s, "k_raw_place", k_raw_place<<<l.grid, 256, 0, s>>>(r, b, cap_hits, status));
  return cudaGetLastError();
}

}  // namespace ptca
