// Export of results and intermediates with event-local input indices (the batch
// stores batch-wide input indices internally).
#include "ptca_internal.cuh"

namespace ptca {

namespace {

__device__ __forceinline__ void to_local(const Buffers& b, int E, const int32_t* src, int32_t* dst,
                                         int32_t* ev) {
  const int e = find_event(b.hit_off, E, src[0]);
  const int32_t off = b.hit_off[e];
#pragma unroll
  for (int k = 0; k < kMaxHits; ++k) dst[k] = src[k] >= 0 ? src[k] - off : -1;
  *ev = e;
}

__global__ void k_export_ntuplets(Buffers b) {
  const uint64_t S = b.cnt[CNT_SV];
  const int E = b.hdr->n_events;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += stride) {
    const uint32_t t = b.ord[b.sv[j]];
    int32_t ev;
    to_local(b, E, b.nt_hits + (uint64_t)t * kMaxHits, b.exp_hits + j * kMaxHits, &ev);
    b.exp_n[j] = b.nt_n[t];
    b.exp_q[j] = b.nt_q[t];
    b.exp_ev[j] = ev;
  }
}

__global__ void k_export_candidates(Buffers b) {
  const uint64_t T = b.cnt[CNT_SCAN_NT];
  const int E = b.hdr->n_events;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride) {
    int32_t ev;
    to_local(b, E, b.nt_hits + t * kMaxHits, b.exp_hits + t * kMaxHits, &ev);
    b.exp_n[t] = b.nt_n[t];
    b.exp_q[t] = b.nt_q[t];
    b.exp_ev[t] = ev;
  }
}

__global__ void k_export_cells(Buffers b, uint64_t cap_cells, int32_t* out3) {
  const uint64_t nc = min(b.cnt[CNT_CELLS], (unsigned long long)cap_cells);
  const int E = b.hdr->n_events;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
    if (b.cell_out[c] == kHole) {
      out3[c * 3 + 0] = out3[c * 3 + 1] = out3[c * 3 + 2] = -1;
      continue;
    }
    const int32_t gi = (int32_t)b.perm[b.cell_in[c]], go = (int32_t)b.perm[b.cell_out[c]];
    const int e = find_event(b.hit_off, E, gi);
    out3[c * 3 + 0] = gi - b.hit_off[e];
    out3[c * 3 + 1] = go - b.hit_off[e];
    out3[c * 3 + 2] = e;
  }
}

__global__ void k_export_links(Buffers b, uint64_t cap_links, int32_t* out4, float* outq,
                               bool gated) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const int E = b.hdr->n_events;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = b.link_src[l];
    if (a == kHole || (gated && !b.gate_keep[l])) continue;  // hole or removed link
    const int32_t g0 = (int32_t)b.perm[b.cell_in[a]], g1 = (int32_t)b.perm[b.cell_out[a]];
    const int32_t g2 = (int32_t)b.perm[b.cell_out[b.link_dst[l]]];
    const int e = find_event(b.hit_off, E, g0);
    const int32_t off = b.hit_off[e];
    out4[l * 4 + 0] = g0 - off;
    out4[l * 4 + 1] = g1 - off;
    out4[l * 4 + 2] = g2 - off;
    out4[l * 4 + 3] = e;
    outq[l] = b.link_q[l];
  }
}

}  // namespace

void launch_export_ntuplets(const Buffers& b, const Launch& l, cudaStream_t s) {
  PT_TRACE(l, s, "k_export_ntuplets", k_export_ntuplets<<<l.grid, 256, 0, s>>>(b));
}
void launch_export_candidates(const Buffers& b, const Launch& l, cudaStream_t s) {
  k_export_candidates<<<l.grid, 256, 0, s>>>(b);
}
void launch_export_cells(const Buffers& b, const Params& p, const Launch& l, int32_t* out3,
                         cudaStream_t s) {
  k_export_cells<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_cells, out3);
}
void launch_export_links(const Buffers& b, const Params& p, const Launch& l, int32_t* out4,
                         float* outq, cudaStream_t s, bool gated) {
  k_export_links<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_links, out4, outq, gated);
}

}  // namespace ptca
