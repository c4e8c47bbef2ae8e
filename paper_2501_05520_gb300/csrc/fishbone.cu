// Fishbone duplicate removal (optional; the library's reading of the overlap cleaning of
// the Patatrack chain, whose steps Sec. 2.2.1 names; the paper gives no detail of it).
//
// A track crossing two overlapping sensors of one layer leaves two hits there, and its
// cells from both to the next hit point the same way.  Active cells (at least one
// outgoing link, after the learned gate when it is set) that end on the same hit are
// compared two by two when their inner hits lie on different layers or on different
// sensors of one layer (radii, barrel, or |z|, disks, more than 0.1 cm apart: the
// stand-in for a sensor identity, which the hit input does not carry).  With u, v the
// float32 vectors from each cell's inner hit to the common outer hit, a pair is aligned
// when u.v > 0 and (u.v)^2 >= 0.99999 |u|^2 |v|^2.
// Of an aligned pair on the same inner layer the shorter cell loses (the longer lever
// arm stays), on different inner layers the longer one (the consecutive-layer cell
// stays); at equal lengths the cell whose inner hit has the larger input index loses.
// A cell that loses to some aligned partner is removed with all its links.  Activity is
// read before anything is removed, so the result does not depend on the order of the
// comparisons: each cell decides only its own fate.
//
// The active cells are the sources of the links (with the gate: of the kept links), so
// they are found from the link slots: the slot that heads a source's out-link list
// stands for its source.  They are grouped by outer
// hit with a counting sort (k_fb_count, a scan, k_fb_scatter, which also writes each
// cell's comparison record), and k_fb_compare takes one active cell per thread and
// compares it with the other records of its group.  The removal
// flags are zeroed for every cell first and set only for the removed ones.
// k_fb_filter_clear / k_fb_filter_set: one thread per link slot; the keep mask of the
//   ntuplet search becomes (gate keep, if any) and neither end removed, and the link
//   flags of the ntuplet search are rebuilt from the kept links (cleared for every end
//   first, then set for the kept ones, in a second launch).
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr float kFbCos2 = 0.99999f;
constexpr float kFbSensorGap = 0.1f;  // cm between two sensors of one layer

// One active cell as the comparisons read it (32 bytes, two float4 in fb_rec).
struct alignas(16) FbCell {
  float4 u;       // outer hit - inner hit (x, y, z), |u|^2
  uint32_t key;   // input index of the inner hit
  uint32_t lay;   // layer of the inner hit
  float sensor;   // the inner hit's radius (barrel) or |z| (disk)
  uint32_t cell;  // the cell
};
static_assert(sizeof(FbCell) == 32, "two float4 per record");

// Does cell a lose to cell c (both ending on the same hit)?  Alignment in float32 with
// correctly rounded operations in a fixed order, no FMA.
__device__ __forceinline__ bool fb_loses(const FbCell& a, const FbCell& c) {
  if (a.lay == c.lay && !(fabsf(fsub(a.sensor, c.sensor)) > kFbSensorGap)) return false;
  const float dot = fadd(fadd(fmul(a.u.x, c.u.x), fmul(a.u.y, c.u.y)), fmul(a.u.z, c.u.z));
  if (!(dot > 0.0f) || !(fmul(dot, dot) >= fmul(kFbCos2, fmul(a.u.w, c.u.w)))) return false;
  if (a.u.w == c.u.w) return a.key > c.key;
  return a.lay == c.lay ? a.u.w < c.u.w : a.u.w > c.u.w;
}

__device__ __forceinline__ FbCell fb_cell(const Buffers& b, float4 ph, uint32_t c, int32_t B) {
  const uint32_t hi = b.cell_in[c];
  const float4 pi = b.hit4[hi];
  FbCell f;
  f.u.x = fsub(ph.x, pi.x);
  f.u.y = fsub(ph.y, pi.y);
  f.u.z = fsub(ph.z, pi.z);
  f.u.w = fadd(fadd(fmul(f.u.x, f.u.x), fmul(f.u.y, f.u.y)), fmul(f.u.z, f.u.z));
  f.key = b.perm[hi];
  f.lay = (b.hbin[hi] / (uint32_t)B) % kLayers;
  f.sensor = f.lay < 4 ? pi.w : fabsf(pi.z);
  f.cell = c;
  return f;
}

// The source of link slot l when l heads an active source's out-link list, else kHole.
__device__ __forceinline__ uint32_t run_source(const Buffers& b, uint64_t l, bool gated) {
  const uint32_t a = b.link_src[l];
  if (a == kHole || b.cell_head[a] != (uint32_t)l) return kHole;
  if (gated && !b.has_out[a]) return kHole;  // no link of the run passed the gate
  return a;
}

__global__ void k_fb_count(Buffers b, uint64_t cap_links, bool gated) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = run_source(b, l, gated);
    if (a != kHole) atomicAdd(&b.fb_cnt[b.cell_out[a]], 1u);
  }
}

__global__ void k_fb_scatter(Buffers b, int32_t B, uint64_t cap_links, bool gated) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = run_source(b, l, gated);
    if (a == kHole) continue;
    const uint32_t h = b.cell_out[a];
    const uint32_t pos = b.fb_start[h] + atomicSub(&b.fb_cnt[h], 1u) - 1u;
    if (!PT_CHECK(b.cnt, pos < cap_links, DBG_FB_RECORD)) continue;
    reinterpret_cast<FbCell*>(b.fb_rec)[pos] = fb_cell(b, b.hit4[h], a, B);
  }
}

// One active cell per thread against the other active cells ending on its outer hit
// (the records of its group, consecutive in fb_rec).
__global__ void k_fb_compare(Buffers b) {
  const uint32_t n_act = b.fb_start[b.cnt[CNT_SCAN_HITS]];
  const uint32_t stride = gridDim.x * blockDim.x;
  const FbCell* rec = reinterpret_cast<const FbCell*>(b.fb_rec);
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_act; p += stride) {
    const FbCell ca = rec[p];
    const uint32_t h = b.cell_out[ca.cell];
    const uint32_t g0 = b.fb_start[h], g1 = b.fb_start[h + 1];
    bool lose = false;
    for (uint32_t q = g0; q < g1 && !lose; ++q)
      if (q != p) lose = fb_loses(ca, rec[q]);
    if (lose) b.fb_kill[ca.cell] = 1;
  }
}

// Keep mask of every link slot: the gate's (gated) and neither end removed; the flags
// of both ends cleared.  The kept links are counted.
__global__ void k_fb_filter_clear(Buffers b, uint64_t cap_links, bool gated) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t kept = 0;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = b.link_src[l];
    bool k = false;
    if (a != kHole) {
      const uint32_t d = b.link_dst[l];
      k = (!gated || b.gate_keep[l]) && !b.fb_kill[a] && !b.fb_kill[d];
      b.has_out[a] = 0;
      b.has_in[d] = 0;
    }
    b.gate_keep[l] = k ? 1 : 0;
    kept += k ? 1u : 0u;
  }
  const unsigned long long tot = __reduce_add_sync(kFull, kept);
  if (lane_id() == 0 && tot) atomicAdd(&b.cnt[CNT_GATE_KEPT], tot);
}

// Flags of the ends of every kept link.
__global__ void k_fb_filter_set(Buffers b, uint64_t cap_links) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    if (!b.gate_keep[l]) continue;
    b.has_out[b.link_src[l]] = 1;
    b.has_in[b.link_dst[l]] = 1;
  }
}

}  // namespace

void launch_fishbone(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                     bool gated) {
  cudaMemsetAsync(&b.cnt[CNT_GATE_KEPT], 0, sizeof(unsigned long long), s);  // recounted
  cudaMemsetAsync(b.fb_kill, 0, (size_t)p.max_cells, s);
  cudaMemsetAsync(b.fb_cnt, 0, (size_t)(p.max_hits + 1) * 4, s);
  PT_TRACE(l, s, "k_fb_count",
           k_fb_count<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_links, gated));
  PT_TRACE(l, s, "scan", launch_scan(b.fb_cnt, b.fb_start, &b.cnt[CNT_SCAN_HITS], b.scan_part, s));
  PT_TRACE(l, s, "k_fb_scatter",
           k_fb_scatter<<<l.grid, 256, 0, s>>>(b, p.phi_bins, (uint64_t)p.max_links, gated));
  PT_TRACE(l, s, "k_fb_compare", k_fb_compare<<<l.grid, 256, 0, s>>>(b));
  PT_TRACE(l, s, "k_fb_filter_clear",
           k_fb_filter_clear<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_links, gated));
  PT_TRACE(l, s, "k_fb_filter_set",
           k_fb_filter_set<<<l.grid, 256, 0, s>>>(b, (uint64_t)p.max_links));
}

}  // namespace ptca
