// Training kernels of the learned gate: mean binary cross-entropy of sigmoid(score)
// against 0/1 labels, its gradient with respect to the 5057 float32 parameters, and an
// Adam update.  Layout of the parameter vector: W1 [64,12], b1 [64], W2 [64,64], b2 [64],
// w3 [64], b3 [1] (row-major), the same as pt_set_gate takes.
//
// k_gate_grad: one 256-thread CTA per block of 128 samples (grid-stride over blocks).
// Two threads per sample run the forward and backward passes over 32 hidden units each,
// keeping the activations and their gradients in shared memory; then the CTA reduces
// the per-sample outer products (dW = sum over samples of dz x h) and adds them to the
// global gradient with one atomic per parameter per block.
#include "ptca_internal.cuh"

namespace ptca {

namespace {

constexpr int kS = 128;                 // samples per block
constexpr int kH = kGateHidden;         // 64
constexpr int kF = kGateFeat;           // 12
constexpr int kOW1 = 0, kOB1 = kOW1 + kH * kF, kOW2 = kOB1 + kH, kOB2 = kOW2 + kH * kH;
constexpr int kOW3 = kOB2 + kH, kOB3 = kOW3 + kH;
constexpr int kWPad = 5060;
constexpr size_t kGradSmem = sizeof(float) * (kWPad + kS * kF + 4 * kS * kH + kS + 4);

__global__ void __launch_bounds__(256)
    k_gate_grad(const float* w, const float* X, const float* y, int64_t n, float* grad,
                float* loss) {
  extern __shared__ float sm[];
  float* sw = sm;
  float* sx = sw + kWPad;
  float* sh1 = sx + kS * kF;
  float* sh2 = sh1 + kS * kH;
  float* sd2 = sh2 + kS * kH;
  float* sd1 = sd2 + kS * kH;
  float* sds = sd1 + kS * kH;
  const int tid = threadIdx.x;
  const int s = tid & (kS - 1), half = tid >> 7;  // sample, which 32 hidden units
  for (int i = tid; i < kGateParams; i += blockDim.x) sw[i] = w[i];
  const float inv_n = 1.0f / (float)n;
  for (int64_t base = (int64_t)blockIdx.x * kS; base < n; base += (int64_t)gridDim.x * kS) {
    __syncthreads();
    const int64_t g = base + s;
    const bool valid = g < n;
    if (half == 0)
      for (int k = 0; k < kF; ++k) sx[s * kF + k] = valid ? X[g * kF + k] : 0.0f;
    __syncthreads();
    // layer 1
    for (int j = half * 32; j < half * 32 + 32; ++j) {
      float z = sw[kOB1 + j];
      for (int k = 0; k < kF; ++k) z += sw[kOW1 + j * kF + k] * sx[s * kF + k];
      sh1[s * kH + j] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    // layer 2
    for (int j = half * 32; j < half * 32 + 32; ++j) {
      float z = sw[kOB2 + j];
      for (int i = 0; i < kH; ++i) z += sw[kOW2 + j * kH + i] * sh1[s * kH + i];
      sh2[s * kH + j] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    // output, loss, d loss / d score
    if (half == 0) {
      float sc = sw[kOB3];
      for (int j = 0; j < kH; ++j) sc += sw[kOW3 + j] * sh2[s * kH + j];
      float ds = 0.0f;
      if (valid) {
        const float yy = y[g];
        const float l = fmaxf(sc, 0.0f) - yy * sc + log1pf(expf(-fabsf(sc)));
        atomicAdd(loss, l * inv_n);
        ds = (1.0f / (1.0f + expf(-sc)) - yy) * inv_n;
      }
      sds[s] = ds;
    }
    __syncthreads();
    for (int j = half * 32; j < half * 32 + 32; ++j)
      sd2[s * kH + j] = sh2[s * kH + j] > 0.0f ? sds[s] * sw[kOW3 + j] : 0.0f;
    __syncthreads();
    for (int i = half * 32; i < half * 32 + 32; ++i) {
      float d = 0.0f;
      if (sh1[s * kH + i] > 0.0f)
        for (int j = 0; j < kH; ++j) d += sd2[s * kH + j] * sw[kOW2 + j * kH + i];
      sd1[s * kH + i] = d;
    }
    __syncthreads();
    // reductions over the block's samples
    for (int e = tid; e < kH * kH; e += blockDim.x) {
      const int j = e / kH, i = e % kH;
      float acc = 0.0f;
      for (int t = 0; t < kS; ++t) acc += sd2[t * kH + j] * sh1[t * kH + i];
      atomicAdd(&grad[kOW2 + e], acc);
    }
    for (int e = tid; e < kH * kF; e += blockDim.x) {
      const int j = e / kF, k = e % kF;
      float acc = 0.0f;
      for (int t = 0; t < kS; ++t) acc += sd1[t * kH + j] * sx[t * kF + k];
      atomicAdd(&grad[kOW1 + e], acc);
    }
    if (tid < kH) {
      float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
      for (int t = 0; t < kS; ++t) {
        g1 += sd1[t * kH + tid];
        g2 += sd2[t * kH + tid];
        g3 += sds[t] * sh2[t * kH + tid];
      }
      atomicAdd(&grad[kOB1 + tid], g1);
      atomicAdd(&grad[kOB2 + tid], g2);
      atomicAdd(&grad[kOW3 + tid], g3);
    } else if (tid == kH) {
      float gb = 0.0f;
      for (int t = 0; t < kS; ++t) gb += sds[t];
      atomicAdd(&grad[kOB3], gb);
    }
  }
}

__global__ void k_gate_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

cudaError_t launch_gate_grad(const float* w, const float* X, const float* y, int64_t n,
                             float* grad, float* loss, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_gate_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kGradSmem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(grad, 0, kGateParams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n + kS - 1) / kS;
  const int grid = (int)(blocks < 2 * sms ? blocks : 2 * sms);
  if (grid > 0) k_gate_grad<<<grid, 256, kGradSmem, s>>>(w, X, y, n, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_gate_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr,
                             float b1, float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_gate_adam<<<(int)((n + 255) / 256), 256, 0, s>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace ptca
