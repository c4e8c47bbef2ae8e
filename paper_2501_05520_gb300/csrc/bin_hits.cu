// Stage A1: load + bin.  Hits of a batch are counting-sorted by (event, layer, phi bin)
// into a (x, y, z, r) float4 array so that the doublet search reads each outer-layer
// azimuthal window as one contiguous range (Sec. 2.2.1, Fig. 2: hits per layer are
// paired with hits of the adjacent layer).  r = sqrt(x*x + y*y) in correctly rounded
// float32; the azimuth is used for binning only, never inside a cut.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// Reset per-batch counters and the histogram / flag arrays, sized from the header.
__global__ void k_clear(Buffers b, int32_t phi_bins) {
  const int E = b.hdr->n_events, N = b.hdr->n_hits;
  const int nb = E * kLayers * phi_bins;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t0; i <= nb; i += stride) b.bin_cnt[i] = 0;
  for (int i = t0; i < E * kLayers; i += stride) {
    b.layer_rmax[i] = 0u;
    b.layer_rmin[i] = 0x7f800000u;  // +inf
    b.layer_zmin[i] = 0xffffffffu;
    b.layer_zmax[i] = 0u;
  }
  for (int i = t0; i <= N; i += stride) b.bucket_cnt[i] = 0;
  for (int i = t0; i < N; i += stride) b.used[i] = 0;
  if (t0 == 0) {
    b.cnt[CNT_CELLS] = 0;
    b.cnt[CNT_LINKS] = 0;
    b.cnt[CNT_NT] = 0;
    b.cnt[CNT_STATUS] = 0;
    b.cnt[CNT_DEBUG_SITE] = 0;
    b.cnt[CNT_GATE_KEPT] = 0;
    b.cnt[CNT_SCAN_NT] = 0;
    b.cnt[CNT_SV] = 0;
    b.cnt[CNT_CELLS_USED] = 0;
    b.cnt[CNT_LINKS_USED] = 0;
    b.cnt[CNT_SCAN_BINS] = (unsigned long long)nb;
    b.cnt[CNT_SCAN_HITS] = (unsigned long long)N;
  }
}

__device__ __forceinline__ float hit_radius(float x, float y) {
  return fsqrt(fadd(fmul(x, x), fmul(y, y)));
}

// Histogram: global bin of every input hit and its rank inside the bin; the r and z
// ranges per (event, layer), reduced within the warp before the atomics.
__global__ void k_bin_count(Buffers b, int32_t B) {
  const int E = b.hdr->n_events, N = b.hdr->n_hits;
  const float scale = (float)B / (2.0f * kPi);
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < N; base += stride) {
    const int g = base + threadIdx.x;
    const bool valid = g < N;
    uint32_t key = 0xffffffffu;  // event*10 + layer
    float r = 0.0f;
    uint32_t zk = 0;
    if (valid) {
      const int L = b.in_layer[g];
      if (L >= kLayers) {
        atomicOr(&b.cnt[CNT_STATUS], ST_LAYER);
        b.in_bin[g] = 0xffffffffu;
      } else {
        const int e = find_event(b.hit_off, E, g);
        const float x = b.in_x[g], y = b.in_y[g];
        r = hit_radius(x, y);
        zk = float_order_key(b.in_z[g]);
        int bin = (int)floorf((atan2f(y, x) + kPi) * scale);
        bin = bin < 0 ? 0 : (bin >= B ? B - 1 : bin);
        key = (uint32_t)(e * kLayers + L);
        const uint32_t gb = key * (uint32_t)B + (uint32_t)bin;
        b.in_bin[g] = gb;
        b.in_rank[g] = atomicAdd(&b.bin_cnt[gb], 1u);
      }
    }
    // per (event, layer) radius range: one atomic each per distinct key in the warp
    const unsigned peers = __match_any_sync(kFull, key);
    // r >= 0, so the integer order of the bit patterns is the float order
    const unsigned m = __reduce_max_sync(peers, __float_as_uint(r));
    const unsigned mn = __reduce_min_sync(peers, __float_as_uint(r));
    const unsigned zmx = __reduce_max_sync(peers, zk);
    const unsigned zmn = __reduce_min_sync(peers, zk);
    if (key != 0xffffffffu && (__ffs(peers) - 1) == lane_id()) {
      atomicMax(&b.layer_rmax[key], m);
      atomicMin(&b.layer_rmin[key], mn);
      atomicMax(&b.layer_zmax[key], zmx);
      atomicMin(&b.layer_zmin[key], zmn);
    }
  }
}

__global__ void k_bin_scatter(Buffers b, float kmax) {
  const int N = b.hdr->n_hits;
  const int stride = gridDim.x * blockDim.x;
  // per event layer: the outer- and inner-radius terms of the azimuthal windows of the
  // doublet search (inner term 0, the widest window, where the bound does not apply)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.hdr->n_events * kLayers; i += stride) {
    const float a = 0.5f * kmax * __uint_as_float(b.layer_rmax[i]);
    b.layer_asin[i] = a >= 0.7f ? __int_as_float(0x7f800000) : asinf(a);
    const float c = 0.5f * kmax * __uint_as_float(b.layer_rmin[i]);
    b.layer_asin_lo[i] = c < 0.7f ? asinf(c) : 0.0f;
  }
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += stride) {
    const uint32_t gb = b.in_bin[g];
    if (gb == 0xffffffffu) continue;
    const uint32_t s = b.bin_start[gb] + b.in_rank[g];
    if (!PT_CHECK(b.cnt, s < (uint32_t)N, DBG_BIN_SCATTER)) continue;
    const float x = b.in_x[g], y = b.in_y[g], z = b.in_z[g];
    b.hit4[s] = make_float4(x, y, z, hit_radius(x, y));
    b.perm[s] = (uint32_t)g;
    b.hbin[s] = gb;
  }
}

// ---------------------------------------------------------------- device scan
constexpr int kScanThreads = 512;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums,
                                                    uint32_t* total) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t ws = lane < (kScanThreads / 32) ? warp_sums[lane] : 0u;
    const uint32_t wi = warp_incl_scan(ws);
    if (lane < (kScanThreads / 32)) warp_sums[lane] = wi - ws;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = warp_sums[w] + inc - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void chunk_of(uint64_t n, uint64_t* lo, uint64_t* hi) {
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  *lo = min(n, per * blockIdx.x);
  *hi = min(n, *lo + per);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(const uint32_t* in, uint32_t* part,
                                                               const unsigned long long* n_dev) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t tot;
  uint64_t lo, hi;
  chunk_of(*n_dev, &lo, &hi);
  uint32_t acc = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) acc += in[i];
  block_excl_scan(acc, ws, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* part, int nparts) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t tot;
  // nparts <= kScanThreads
  const uint32_t v = threadIdx.x < nparts ? part[threadIdx.x] : 0u;
  const uint32_t ex = block_excl_scan(v, ws, &tot);
  if (threadIdx.x < nparts) part[threadIdx.x] = ex;
  if (threadIdx.x == 0) part[nparts] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const uint32_t* in, uint32_t* out,
                                                             const uint32_t* part,
                                                             const unsigned long long* n_dev) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t tot;
  const uint64_t n = *n_dev;
  uint64_t lo, hi;
  chunk_of(n, &lo, &hi);
  uint32_t carry = part[blockIdx.x];
  for (uint64_t base = lo; base < hi; base += kScanThreads) {
    const uint64_t i = base + threadIdx.x;
    const uint32_t v = i < hi ? in[i] : 0u;
    const uint32_t ex = block_excl_scan(v, ws, &tot);
    if (i < hi) out[i] = carry + ex;
    carry += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

}  // namespace

void launch_scan(const uint32_t* in, uint32_t* out, const unsigned long long* n_dev,
                 uint32_t* part, cudaStream_t s) {
  k_scan_partial<<<kScanBlocks, kScanThreads, 0, s>>>(in, part, n_dev);
  k_scan_top<<<1, kScanThreads, 0, s>>>(part, kScanBlocks);
  k_scan_final<<<kScanBlocks, kScanThreads, 0, s>>>(in, out, part, n_dev);
}

void launch_clear(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  PT_TRACE(l, s, "k_clear", k_clear<<<l.grid, 256, 0, s>>>(b, p.phi_bins));
}

void launch_bin_hits(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s) {
  PT_TRACE(l, s, "k_bin_count", k_bin_count<<<l.grid, 256, 0, s>>>(b, p.phi_bins));
  PT_TRACE(l, s, "scan", launch_scan(b.bin_cnt, b.bin_start, &b.cnt[CNT_SCAN_BINS], b.scan_part, s));
  PT_TRACE(l, s, "k_bin_scatter", k_bin_scatter<<<l.grid, 256, 0, s>>>(b, p.cuts.kmax));
}

namespace {
__global__ void k_debug_inject(Buffers b, unsigned site) {
#ifdef PT_DEBUG
  debug_fail(b.cnt, site);
#endif
}
}  // namespace

cudaError_t launch_debug_inject(const Buffers& b, unsigned site, cudaStream_t s) {
  k_debug_inject<<<1, 1, 0, s>>>(b, site);
  return cudaGetLastError();
}

}  // namespace ptca
