// Learned link gate (optional stage after the cellular-automaton links): every accepted
// link (h0 -> h1 -> h2) gets 12 geometric features (computed from its three hits by the
// link stage's target pass, one bf16 row per link slot), a 12 -> 64 -> 64 -> 1 MLP scores
// it on the tensor cores, and
// links scoring below the threshold are skipped by the ntuplet search: the MLP's
// epilogue sets the in/out flags of the cells of kept links only.  It plays the role of the edge-filtering MLP of the paper's ML
// pipeline (Sec. 2.2.2: an MLP scores graph edges, a fixed threshold removes clearly
// fake ones); the exact cuts stay in force, the gate only removes links.
//
// Features (float32 from the hit coordinates, rounded to bf16 for the MMA):
//   C1, C2 and C3 cut ratios, t_a / cotmax, 10 (t_b - t_a), r0/16, r1/16, r2/16,
//   (z0 - r0 t_a) / z0max, layer0/9, layer1/9, layer2/9; padded with 4 zeros to K = 16.
//
// Tensor-core MLP (128-thread CTAs, six per SM, persistent over 128-link tiles; each
// tile's rows are loaded into registers while the tile before it is computed):
//   D1[128x64] = X[128x16] * W1^T      one tcgen05.mma (M=128, N=64, K=16), TMEM cols 0..63
//   H1 = bf16(relu(D1 + b1))           tcgen05.ld by each warp's 32 TMEM lanes -> smem
//   D2[128x64] = H1[128x64] * W2^T     four tcgen05.mma (K=16 each), the same TMEM columns
//                                      (D1 has been read by then)
//   score = relu(D2 + b2) . w3 + b3    tcgen05.ld + float32 dot in registers
// Operands are bf16 in shared memory in the no-swizzle K-major layout of 8x8 core
// matrices (16 bytes per row, 128 bytes per core matrix; LBO = 128 bytes between core
// matrices along K, SBO = K/8 * 128 bytes between groups of 8 rows).  One thread issues
// the MMAs and commits them to an mbarrier; every wait on it is bounded and sets an
// error flag instead of hanging.
#include <cuda_bf16.h>

#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kTileM = 128;
constexpr uint32_t kIdesc = (1u << 4)                          // D: float32
                            | (1u << 7) | (1u << 10)            // A, B: bf16
                            | ((uint32_t)(kGateHidden >> 3) << 17)  // N = 64
                            | ((uint32_t)(kTileM >> 4) << 24);     // M = 128
constexpr long long kWaitCycles = 1ll << 31;  // ~1 s at 2 GHz: the teardown's limit

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start, LBO, SBO (bytes, >> 4), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

// Bounded wait for the mbarrier phase `parity` to complete; false once `limit` cycles
// have passed.  The limit is checked before every try (try_wait itself may suspend the
// thread for a while), so even a limit of one cycle gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    if (clock64() - t0 >= limit) return false;
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
}

// 32 consecutive TMEM columns of this warp's 32 lanes -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory layout of the MLP kernel (bytes).
constexpr int kOffX = 0;              // 128 x 16 bf16, SBO 256
constexpr int kOffW1 = 4096;          // 64 x 16 bf16, SBO 256
constexpr int kOffW2 = 6144;          // 64 x 64 bf16, SBO 1024
constexpr int kOffH1 = 14336;         // 128 x 64 bf16, SBO 1024
constexpr int kOffF = 30720;          // b1, b2, w3 (64 each), b3, tau
constexpr int kOffBar = 31744;        // mbarrier
constexpr int kOffTmem = 31752;       // TMEM base address
constexpr int kOffFlag = 31756;       // wait status
constexpr int kMlpSmem = 32 * 1024;   // requested: six CTAs per SM by shared memory
constexpr int kMlpCtasPerSm = 6;
constexpr int kMlpTmemCols = 64;      // D1, then D2
static_assert(kMlpCtasPerSm * kMlpTmemCols <= 512, "every resident CTA gets its TMEM columns");
static_assert(kMlpCtasPerSm * (kMlpSmem + 1024) <= 228 * 1024, "six CTAs fit an SM");

// PIPE = true: rows are link slots of the batch, whose bf16 feature rows the link stage
// wrote to gate_x; kept links set the flags the ntuplet search reads.
// PIPE = false: rows are given bf16 feature rows X (standalone scoring).
template <bool PIPE>
__global__ void __launch_bounds__(kTileM, kMlpCtasPerSm)
    k_gate_mlp(const GateWeights* gw, Buffers b, pt_cuts cuts, int32_t B, const uint16_t* X,
               const unsigned long long* n_dev, int64_t n_max, float* score, uint8_t* keep,
               unsigned long long* status, unsigned long long* kept, long long wait_limit) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  float* sb1 = (float*)(sm + kOffF);
  float* sb2 = sb1 + kGateHidden;
  float* sw3 = sb2 + kGateHidden;
  float* sc = sw3 + kGateHidden;
  uint64_t* mbar = (uint64_t*)(sm + kOffBar);
  uint32_t* tslot = (uint32_t*)(sm + kOffTmem);
  volatile uint32_t* flag = (volatile uint32_t*)(sm + kOffFlag);
  // rows: n_max, or the device count clamped to n_max
  const uint64_t n = n_dev ? min((uint64_t)*n_dev, (uint64_t)n_max) : (uint64_t)n_max;

  // weights -> shared memory (already in the operand layout)
  {
    const uint4* w1 = (const uint4*)gw->w1;
    const uint4* w2 = (const uint4*)gw->w2;
    ((uint4*)(sm + kOffW1))[tid] = w1[tid];  // 128 x 16 B
#pragma unroll
    for (int i = 0; i < 4; ++i) ((uint4*)(sm + kOffW2))[tid + 128 * i] = w2[tid + 128 * i];
    if (tid < kGateHidden) {
      sb1[tid] = gw->b1[tid];
      sb2[tid] = gw->b2[tid];
      sw3[tid] = gw->w3[tid];
    }
    if (tid == 0) {
      sc[0] = gw->b3;
      sc[1] = gw->tau;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      *flag = 0;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t ax = smem_u32(sm + kOffX), aw1 = smem_u32(sm + kOffW1);
  const uint32_t aw2 = smem_u32(sm + kOffW2), ah1 = smem_u32(sm + kOffH1);
  uint32_t phase = 0;
  bool pending = false;  // an MMA group was committed and not yet seen complete
  const uint64_t n_tiles = (n + kTileM - 1) / kTileM;

  // this thread's row of tile tt: its source cell (pipeline form) and bf16 feature row
  auto load_row = [&](uint64_t tt, uint4& lo, uint4& hi, uint32_t& src) {
    const uint64_t r = tt * kTileM + tid;
    lo = make_uint4(0, 0, 0, 0);
    hi = lo;
    src = kHole;
    if (tt >= n_tiles || r >= n) return;
    if (PIPE) {
      src = b.link_src[r];
      if (src == kHole) return;
    }
    const uint4* srcp = (const uint4*)((PIPE ? b.gate_x : X) + r * kGateK1);
    lo = srcp[0];
    hi = srcp[1];
  };
  uint4 nlo, nhi;
  uint32_t nsrc;
  load_row(blockIdx.x, nlo, nhi, nsrc);
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint64_t row = t * kTileM + tid;
    // X row -> core-matrix layout: k 0..7 at +0, k 8..15 at +128 within the row group
    unsigned char* xr = sm + kOffX + (tid >> 3) * 256 + (tid & 7) * 16;
    const uint32_t src_cell = nsrc;
    *(uint4*)xr = nlo;
    *(uint4*)(xr + 128) = nhi;
    load_row(t + gridDim.x, nlo, nhi, nsrc);  // in flight while this tile is computed
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
      mma_bf16(tmem, smem_desc(ax, 128, 256), smem_desc(aw1, 128, 256), 0u);
      mma_commit(mbar);
      pending = true;
      if (!mbar_wait(mbar, phase, wait_limit)) *flag = 1;
      else pending = false;
    }
    __syncthreads();
    if (*flag) break;
    phase ^= 1u;
    tc_after_sync();
    // epilogue 1: this thread's row of D1 -> relu(+b1) -> bf16 -> H1 (shared memory)
    {
      unsigned char* hr = sm + kOffH1 + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float v[32];
        tmem_ld32(tmem + lane_base + 32 * half, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {  // 4 core matrices of 8 columns per half
          const int j0 = 32 * half + 8 * c;
          uint4 pk;
          pk.x = pack_bf16x2(fmaxf(v[8 * c + 0] + sb1[j0 + 0], 0.f), fmaxf(v[8 * c + 1] + sb1[j0 + 1], 0.f));
          pk.y = pack_bf16x2(fmaxf(v[8 * c + 2] + sb1[j0 + 2], 0.f), fmaxf(v[8 * c + 3] + sb1[j0 + 3], 0.f));
          pk.z = pack_bf16x2(fmaxf(v[8 * c + 4] + sb1[j0 + 4], 0.f), fmaxf(v[8 * c + 5] + sb1[j0 + 5], 0.f));
          pk.w = pack_bf16x2(fmaxf(v[8 * c + 6] + sb1[j0 + 6], 0.f), fmaxf(v[8 * c + 7] + sb1[j0 + 7], 0.f));
          *(uint4*)(hr + (j0 >> 3) * 128) = pk;
        }
      }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        mma_bf16(tmem, smem_desc(ah1 + 256 * j, 128, 1024), smem_desc(aw2 + 256 * j, 128, 1024),
                 j > 0 ? 1u : 0u);
      mma_commit(mbar);
      pending = true;
      if (!mbar_wait(mbar, phase, wait_limit)) *flag = 1;
      else pending = false;
    }
    __syncthreads();
    if (*flag) break;
    phase ^= 1u;
    tc_after_sync();
    // epilogue 2: relu(D2 + b2) . w3 + b3
    float acc = sc[0];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[32];
      tmem_ld32(tmem + lane_base + 32 * half, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc += fmaxf(v[i] + sb2[32 * half + i], 0.f) * sw3[32 * half + i];
    }
    // pipeline form (src != NULL): row = link slot; kept links set the flags the
    // ntuplet search reads (a link slot that is a hole is never kept)
    bool kp = row < n && acc >= sc[1];
    if (row < n) {
      if (PIPE) {
        if (src_cell == kHole) {
          kp = false;
        } else if (kp) {
          b.has_in[b.link_dst[row]] = 1;
          b.has_out[src_cell] = 1;
        }
      }
      score[row] = acc;
      if (keep) keep[row] = kp ? 1 : 0;
    }
    if (kept) {
      const unsigned bal = __ballot_sync(kFull, kp);
      if ((tid & 31) == 0 && bal) atomicAdd(kept, (unsigned long long)__popc(bal));
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
  }
  // teardown: report a timeout, let an MMA still in flight finish (bounded by the full
  // limit whatever the step waits used), and only then free TMEM
  if (tid == 0 && *flag) {
    atomicOr(status, ST_GATE_TIMEOUT);
    if (pending) mbar_wait(mbar, phase, kWaitCycles);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// float32 features of every current link (gated form: kept links only), row = link slot.
__global__ void k_gate_features_f32(Buffers b, pt_cuts cuts, int32_t B, uint64_t cap_links,
                                    bool gated, float* out) {
  const uint64_t nl = min(b.cnt[CNT_LINKS], (unsigned long long)cap_links);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
    const uint32_t a = b.link_src[l];
    if (a == kHole || (gated && !b.gate_keep[l])) continue;
    const uint32_t h0 = b.cell_in[a], h1 = b.cell_out[a];
    const uint32_t h2 = b.cell_out[b.link_dst[l]];
    float f[kGateFeat];
    gate_link_features(cuts, b.hit4[h0], b.hit4[h1], b.hit4[h2], (b.hbin[h0] / B) % kLayers,
                       (b.hbin[h1] / B) % kLayers, (b.hbin[h2] / B) % kLayers, f);
#pragma unroll
    for (int k = 0; k < kGateFeat; ++k) out[l * kGateFeat + k] = f[k];
  }
}

// float32 feature rows -> bf16 rows padded to 16.
__global__ void k_gate_pack(const float* feat, int64_t n, uint16_t* X) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    float f[kGateFeat];
#pragma unroll
    for (int k = 0; k < kGateFeat; ++k) f[k] = feat[r * kGateFeat + k];
    store_gate_row(X + r * kGateK1, f);
  }
}

}  // namespace

cudaError_t gate_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_gate_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMlpSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gate_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMlpSmem);
  return e;
}

void launch_gate(const Buffers& b, const Params& p, const Launch& l, const GateWeights* w,
                 cudaStream_t s) {
  PT_TRACE(l, s, "k_gate_mlp",
           k_gate_mlp<true><<<l.sms * kMlpCtasPerSm, kTileM, kMlpSmem, s>>>(
               w, b, p.cuts, p.phi_bins, nullptr, &b.cnt[CNT_LINKS], p.max_links, b.gate_score,
               b.gate_keep, &b.cnt[CNT_STATUS], &b.cnt[CNT_GATE_KEPT], p.wait_cycles));
}

void launch_gate_score(const GateWeights* w, const float* feat, int64_t n, float* out,
                       uint16_t* xbuf, unsigned long long* status, int sms, long long wait_cycles,
                       cudaStream_t s) {
  k_gate_pack<<<sms * 4, 256, 0, s>>>(feat, n, xbuf);
  k_gate_mlp<false><<<sms * kMlpCtasPerSm, kTileM, kMlpSmem, s>>>(w, Buffers{}, pt_cuts{}, 1, xbuf, nullptr, n,
                                                        out, nullptr, status, nullptr, wait_cycles);
}

void launch_export_link_features(const Buffers& b, const Params& p, const Launch& l, bool gated,
                                 float* out, cudaStream_t s) {
  k_gate_features_f32<<<l.grid, 256, 0, s>>>(b, p.cuts, p.phi_bins, (uint64_t)p.max_links, gated,
                                              out);
}

}  // namespace ptca
