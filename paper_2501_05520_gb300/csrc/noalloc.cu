// pt_find_doublets_noalloc: the doublet search of one event with all of its scratch in
// a fixed array compiled into the library, for callers that must not allocate device
// memory (see pt_ca.h).  It reuses the library's binning kernels on a view of that
// array and runs its own doublet kernel, which writes the pairs straight into the
// caller's output arrays instead of the context's cell arrays.
#include <string>

#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int64_t kNaMaxHits = 65536;  // largest event accepted
constexpr int kNaBins = 256;           // azimuthal bins per layer
constexpr size_t kNaAlign = 256;

constexpr size_t na_round(size_t x) { return (x + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaNb = (size_t)kLayers * kNaBins + 1;
// Bytes of each scratch buffer, in the order na_layout carves them.
enum NaPart {
  NA_HDR, NA_CNT, NA_OFF, NA_IN_BIN, NA_IN_RANK, NA_HIT4, NA_PERM, NA_HBIN, NA_BIN_CNT,
  NA_BIN_START, NA_RMAX, NA_ASIN, NA_RMIN, NA_ASIN_LO, NA_ZMIN, NA_ZMAX, NA_BUCKET_CNT, NA_USED,
  NA_SCAN,
  NA_PARTS
};
constexpr size_t kNaPart[NA_PARTS] = {
    sizeof(BatchHeader), CNT_N * 8, 2 * 4,                   // header, counters, offsets
    kNaMaxHits * 4, kNaMaxHits * 4,                          // in_bin, in_rank
    kNaMaxHits * 16, kNaMaxHits * 4, kNaMaxHits * 4,         // hit4, perm, hbin
    kNaNb * 4, kNaNb * 4, kLayers * 4, kLayers * 4,          // bins, layer r max, layer asin
    kLayers * 4, kLayers * 4,                                // layer r min, its asin
    kLayers * 4, kLayers * 4,                                // layer z min, max
    (kNaMaxHits + 1) * 4, kNaMaxHits,                        // cleared: bucket, used
    (kScanBlocks + 1) * 4};                                  // scan partials
constexpr size_t na_offset(int part) {
  size_t off = 0;
  for (int i = 0; i < part; ++i) off += na_round(kNaPart[i]);
  return off;
}
constexpr size_t kNaBytes = na_offset(NA_PARTS);

// The scratch.  Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kNaBytes];

// Carves the scratch (device address `base`) into the buffers the binning kernels use.
Buffers na_layout(char* base, const float* x, const float* y, const float* z,
                  const uint8_t* layer) {
  auto at = [&](int part) { return base + na_offset(part); };
  Buffers b{};
  b.hdr = (BatchHeader*)at(NA_HDR);
  b.cnt = (unsigned long long*)at(NA_CNT);
  b.hit_off = (int32_t*)at(NA_OFF);
  b.in_bin = (uint32_t*)at(NA_IN_BIN);
  b.in_rank = (uint32_t*)at(NA_IN_RANK);
  b.hit4 = (float4*)at(NA_HIT4);
  b.perm = (uint32_t*)at(NA_PERM);
  b.hbin = (uint32_t*)at(NA_HBIN);
  b.bin_cnt = (uint32_t*)at(NA_BIN_CNT);
  b.bin_start = (uint32_t*)at(NA_BIN_START);
  b.layer_rmax = (uint32_t*)at(NA_RMAX);
  b.layer_asin = (float*)at(NA_ASIN);
  b.layer_rmin = (uint32_t*)at(NA_RMIN);
  b.layer_asin_lo = (float*)at(NA_ASIN_LO);
  b.layer_zmin = (uint32_t*)at(NA_ZMIN);
  b.layer_zmax = (uint32_t*)at(NA_ZMAX);
  b.bucket_cnt = (uint32_t*)at(NA_BUCKET_CNT);
  b.used = (uint8_t*)at(NA_USED);
  b.scan_part = (uint32_t*)at(NA_SCAN);
  b.in_x = (float*)x;
  b.in_y = (float*)y;
  b.in_z = (float*)z;
  b.in_layer = (uint8_t*)layer;
  return b;
}

__global__ void k_na_header(Buffers b, int32_t n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    b.hdr->n_events = 1;
    b.hdr->n_hits = n;
    b.hit_off[0] = 0;
    b.hit_off[1] = n;
  }
}

// Doublet search of the binned event: one warp per inner hit, the same azimuthal
// window and exact cuts as the batched doublet stage; each accepted pair is written as
// (inner, outer) input indices at a slot taken with one atomic per warp iteration.
__global__ void k_na_doublets(Buffers b, pt_cuts cuts, PairTable pt, int32_t* inner,
                              int32_t* outer, int64_t cap) {
  constexpr float kTwoPi = 6.28318530717958647692f;
  constexpr float kHalfPi = 1.57079632679489661923f;
  const int lane = lane_id();
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t n_sorted = b.bin_start[kLayers * kNaBins];
  const float bins_per_rad = (float)kNaBins / kTwoPi;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_sorted;
       s += nwarps) {
    const uint32_t gb = b.hbin[s];
    const int L = gb / kNaBins, bin = gb - L * kNaBins;
    const float4 hi = b.hit4[s];
    for (int k = 0; k < pt.n_outer[L]; ++k) {
      const int Lo = pt.outer[L][k];
      const float ro_max = __uint_as_float(b.layer_rmax[Lo]);
      if (!(ro_max > hi.w)) continue;
      const float a = 0.5f * cuts.kmax * ro_max;
      const float win = a >= 0.7f ? kHalfPi + 1e-3f
                                  : fminf(asinf(a) - asinf(fminf(0.5f * cuts.kmax * hi.w, a)) + 1e-4f,
                                          kHalfPi + 1e-3f);
      const int w = (int)ceilf(win * bins_per_rad) + 1;
      const uint32_t base = (uint32_t)Lo * kNaBins;
      uint32_t r[4] = {0, 0, 0, 0};
      if (2 * w + 1 >= kNaBins) {
        r[0] = b.bin_start[base];
        r[1] = b.bin_start[base + kNaBins];
      } else if (bin - w < 0) {
        r[0] = b.bin_start[base + kNaBins + bin - w];
        r[1] = b.bin_start[base + kNaBins];
        r[2] = b.bin_start[base];
        r[3] = b.bin_start[base + bin + w + 1];
      } else if (bin + w >= kNaBins) {
        r[0] = b.bin_start[base + bin - w];
        r[1] = b.bin_start[base + kNaBins];
        r[2] = b.bin_start[base];
        r[3] = b.bin_start[base + bin + w - kNaBins + 1];
      } else {
        r[0] = b.bin_start[base + bin - w];
        r[1] = b.bin_start[base + bin + w + 1];
      }
      for (int part = 0; part < 2; ++part) {
        for (uint32_t o0 = r[2 * part]; o0 < r[2 * part + 1]; o0 += 32) {
          const uint32_t o = o0 + lane;
          const bool pass = o < r[2 * part + 1] && doublet_pass(cuts, hi, b.hit4[o]);
          const unsigned bal = __ballot_sync(kFull, pass);
          if (bal == 0) continue;
          unsigned long long slot = 0;
          if (lane == 0) slot = atomicAdd(&b.cnt[CNT_CELLS], (unsigned long long)__popc(bal));
          slot = __shfl_sync(kFull, slot, 0) + __popc(bal & lt_mask);
          if (pass && slot < (unsigned long long)cap) {
            inner[slot] = (int32_t)b.perm[s];
            outer[slot] = (int32_t)b.perm[o];
          }
        }
      }
    }
  }
}

pt_status na_fail(pt_status st, const char* msg, cudaError_t e = cudaSuccess) {
  std::string m = msg;
  if (e != cudaSuccess) {
    m += ": ";
    m += cudaGetErrorString(e);
  }
  set_last_error(m.c_str());
  return st;
}

}  // namespace

}  // namespace ptca

using namespace ptca;

extern "C" pt_status pt_find_doublets_noalloc(const pt_cuts* cuts, int64_t n, const float* x,
                                              const float* y, const float* z,
                                              const uint8_t* layer, int32_t* inner,
                                              int32_t* outer, int64_t cap, int64_t* n_out,
                                              void* stream) {
  set_last_error("");
  if (!cuts || !n_out) return na_fail(PT_ERR_INVALID, "cuts and n_out must not be NULL");
  if (n < 0 || n > kNaMaxHits)
    return na_fail(PT_ERR_CAPACITY, "pt_find_doublets_noalloc accepts at most 65536 hits");
  if (cap < 0) return na_fail(PT_ERR_INVALID, "cap must be >= 0");
  if (n > 0 && (!x || !y || !z || !layer))
    return na_fail(PT_ERR_INVALID, "hit arrays must not be NULL");
  if (cap > 0 && (!inner || !outer))
    return na_fail(PT_ERR_INVALID, "output arrays must not be NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PT_ERR_CUDA, "cudaGetDevice failed", e);
  // The scratch array's device address on the current device, looked up on every call
  // (with the device current) so that a context made again after a reset is followed.
  void* base = nullptr;
  e = cudaGetSymbolAddress(&base, g_scratch);
  if (e != cudaSuccess || !base)
    return na_fail(PT_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed", e);
  cudaStream_t s = (cudaStream_t)stream;
  Buffers b = na_layout((char*)base, x, y, z, layer);
  Params p{};
  p.cuts = *cuts;
  p.phi_bins = kNaBins;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_fail(PT_ERR_CUDA, "cannot query the multiprocessor count", e);
  Launch l{sms, sms * 4, sms * 5};
  k_na_header<<<1, 32, 0, s>>>(b, (int32_t)n);
  launch_clear(b, p, l, s);  // zeroes the counters and histograms the last call left
  launch_bin_hits(b, p, l, s);
  k_na_doublets<<<sms * 4, 256, 0, s>>>(b, *cuts, default_pair_table(), inner, outer, cap);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PT_ERR_CUDA, "kernel launch failed", e);
  unsigned long long cnt[CNT_N];
  e = cudaMemcpyAsync(cnt, b.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(PT_ERR_CUDA, "reading the result count failed", e);
  *n_out = (int64_t)cnt[CNT_CELLS];
  if (cnt[CNT_STATUS] & ST_LAYER) return na_fail(PT_ERR_INVALID, "layer code > 9 in input");
  if ((int64_t)cnt[CNT_CELLS] > cap)
    return na_fail(PT_ERR_CAPACITY, "output capacity too small; *n_out holds the needed size");
  return PT_OK;
}
