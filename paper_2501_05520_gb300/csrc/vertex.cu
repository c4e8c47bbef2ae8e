// Primary vertices of the fitted tracks (Sec. 2.2.1: vertex reconstruction is the last
// of Patatrack's sub-algorithms, and the chain returns the reconstructed tracks and
// vertices, Fig. 2).  The paper gives no algorithm; the library's reading:
//   [V1] an event's tracks with at least min_hits hits and a finite z0 take part;
//   [V2] they are ordered by z0 (ties: position in the event's canonical track order)
//        and the ordered list is cut where the float32 step to the next z0 exceeds dz
//        (single-linkage clustering in z0);
//   [V3] every group of at least two tracks is a vertex: z = mean z0, sum of pT^2,
//        number of tracks; vertices in order of z; every used track records its vertex.
//
// One block of 1024 threads per event.  The selected tracks' (z0, position) keys are
// sorted in shared memory (bitonic, up to 16384 per event); each group start finds its
// group's end by walking forward, a block scan numbers the groups of two or more, and
// each vertex is summed in z order by one thread (float32).  The vertices of event e go
// to a staging area at floor(t0 / 2) (an event with T tracks has at most T / 2
// vertices); a scan over the events' vertex counts and one more kernel place them in
// one batch-wide list and turn each track's vertex into a batch-wide index.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kVtxThreads = 1024;
constexpr int kVtxMax = 16384;                    // selected tracks per event
constexpr int kVtxPer = kVtxMax / kVtxThreads;    // scan elements per thread
constexpr size_t kVtxSmem = (size_t)kVtxMax * 12;  // keys (8 bytes) + scan array (4 bytes)

// float -> unsigned key with the same order (negative below positive)
__device__ __forceinline__ uint32_t ord_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// In-place exclusive scan of a[0..kVtxMax) (kVtxPer consecutive entries per thread);
// returns the total.  All threads of the block take part.
__device__ uint32_t vtx_block_scan(uint32_t* a, uint32_t* warp_tot) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t loc[kVtxPer];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kVtxPer; ++i) {
    loc[i] = a[t * kVtxPer + i];
    s += loc[i];
  }
  const uint32_t inc = warp_incl_scan(s);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t x = warp_tot[lane];
    const uint32_t xi = warp_incl_scan(x);
    warp_tot[lane] = xi - x;
    if (lane == 31) warp_tot[32] = xi;
  }
  __syncthreads();
  uint32_t run = warp_tot[w] + inc - s;
#pragma unroll
  for (int i = 0; i < kVtxPer; ++i) {
    a[t * kVtxPer + i] = run;
    run += loc[i];
  }
  const uint32_t total = warp_tot[32];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kVtxThreads) k_vertex_event(Buffers b, int32_t min_hits,
                                                              float dz, uint64_t cap_nt) {
  extern __shared__ unsigned char vsm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(vsm);  // [kVtxMax]
  uint32_t* vf = reinterpret_cast<uint32_t*>(vsm + (size_t)kVtxMax * 8);  // [kVtxMax]
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t s_n;
  const int e = blockIdx.x, tid = threadIdx.x;
  if (e == 0 && tid == 0) b.cnt[CNT_SCAN_EV] = (unsigned long long)gridDim.x;
  // the event's tracks, clamped to the cleaned ntuplets of the batch
  const int64_t S = (int64_t)min(b.cnt[CNT_SV], (unsigned long long)cap_nt);
  const int64_t t0 = min(max(b.ev_nt_off[e], (int64_t)0), S);
  const int64_t nt = min(max(b.ev_nt_off[e + 1], t0), S) - t0;
  if (tid == 0) s_n = 0;
  __syncthreads();
  // [V1] the tracks that take part, keyed by (z0, position)
  for (int64_t i = tid; i < nt; i += kVtxThreads) {
    const pt_track& tr = b.tracks[t0 + i];
    const float z0 = tr.z0;
    b.trk_vtx[t0 + i] = -1;
    if ((int)tr.nhits >= min_hits && isfinite(z0)) {
      const uint32_t k = atomicAdd(&s_n, 1u);
      if (k < (uint32_t)kVtxMax) key[k] = ((unsigned long long)ord_f32(z0) << 32) | (uint32_t)i;
    }
  }
  __syncthreads();
  const uint32_t n = s_n;
  if (n > (uint32_t)kVtxMax) {
    if (tid == 0) {
      atomicOr(&b.cnt[CNT_STATUS], ST_VTX);
      b.ev_nv[e] = 0;
    }
    return;
  }
  // [V2] bitonic sort of the keys, padded to a power of two
  uint32_t P = 1;
  while (P < n) P <<= 1;
  for (uint32_t i = n + tid; i < P; i += kVtxThreads) key[i] = ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < P; i += kVtxThreads) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const unsigned long long a = key[i], c = key[l];
          if ((a > c) == ((i & k) == 0)) {
            key[i] = c;
            key[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  auto zk = [&](uint32_t k) { return unord_f32((uint32_t)(key[k] >> 32)); };
  auto starts = [&](uint32_t k) { return k == 0 || fsub(zk(k), zk(k - 1)) > dz; };
  // a group start whose group holds at least two tracks marks a vertex
  for (uint32_t k = tid; k < (uint32_t)kVtxMax; k += kVtxThreads) {
    uint32_t f = 0;
    if (k < n && starts(k)) f = k + 1 < n && !starts(k + 1);
    vf[k] = f;
  }
  __syncthreads();
  const uint32_t nv = vtx_block_scan(vf, warp_tot);
  // [V3] each vertex summed in z order; its tracks record it
  const int64_t vbase = t0 / 2;
  for (uint32_t k = tid; k < n; k += kVtxThreads) {
    const bool is_v = (k + 1 < n ? vf[k + 1] : nv) > vf[k];
    if (!is_v) continue;
    const uint32_t v = vf[k];
    uint32_t end = k + 1;  // the group is [k, end)
    while (end < n && !starts(end)) ++end;
    float zs = 0.0f, p2 = 0.0f;
#pragma unroll 8
    for (uint32_t m = k; m < end; ++m) {  // the loads of eight tracks in flight at once
      const uint32_t i = (uint32_t)key[m];
      const float pt = b.tracks[t0 + i].pt;
      zs = fadd(zs, zk(m));
      p2 = fadd(p2, fmul(pt, pt));
      b.trk_vtx[t0 + i] = (int32_t)v;
    }
    pt_vertex out;
    out.z = fdiv(zs, (float)(end - k));
    out.sum_pt2 = p2;
    out.n_tracks = (int32_t)(end - k);
    out.event = e;
    b.vtx_stage[vbase + v] = out;
  }
  if (tid == 0) b.ev_nv[e] = nv;
}

// Event e's vertices to the batch-wide list at ev_v_scan[e]; its tracks' vertices
// become batch-wide indices; per-event offsets as int64 and the total count.
__global__ void k_vertex_compact(Buffers b, uint64_t cap_nt) {
  const int e = blockIdx.x, E = gridDim.x;
  const int64_t S = (int64_t)min(b.cnt[CNT_SV], (unsigned long long)cap_nt);
  const int64_t t0 = min(max(b.ev_nt_off[e], (int64_t)0), S);
  const int64_t t1 = min(max(b.ev_nt_off[e + 1], t0), S);
  const uint32_t v0 = b.ev_v_scan[e], nv = b.ev_nv[e];
  for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) b.vtx[v0 + v] = b.vtx_stage[t0 / 2 + v];
  for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int32_t v = b.trk_vtx[t];
    if (v >= 0) b.trk_vtx[t] = v + (int32_t)v0;
  }
  if (e == 0)
    for (int i = threadIdx.x; i <= E; i += blockDim.x) b.ev_vtx_off[i] = (int64_t)b.ev_v_scan[i];
  if (e == 0 && threadIdx.x == 0) b.cnt[CNT_VTX] = b.ev_v_scan[E];
}

}  // namespace

cudaError_t launch_vertices(const Buffers& b, int n_events, int32_t min_hits, float dz,
                            uint64_t cap_nt, const Launch& l, cudaStream_t s) {
  if (n_events < 1) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(k_vertex_event,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVtxSmem);
  if (err != cudaSuccess) return err;
  PT_TRACE(l, s, "k_vertex_event",
           k_vertex_event<<<n_events, kVtxThreads, kVtxSmem, s>>>(b, min_hits, dz, cap_nt));
  PT_TRACE(l, s, "scan", launch_scan(b.ev_nv, b.ev_v_scan, &b.cnt[CNT_SCAN_EV], b.scan_part, s));
  PT_TRACE(l, s, "k_vertex_compact", k_vertex_compact<<<n_events, 256, 0, s>>>(b, cap_nt));
  return cudaGetLastError();
}

}  // namespace ptca
