// kpz_mlp.cu -- the learned surrogate: a 4-128-128-128-1 GELU MLP with
// bfloat16 weights and float32 arithmetic, trained with Adam by the kernels
// below (forward, backward, gradient reduction, update).
//
// The paper has no learned component. The network maps the features of a
// realisation and a time (log2 L, log t, p, q, scaled) to log W^2; the
// ensemble batcher uses its curves to estimate saturation times. Parameters
// are one flat vector: W1 (128x4 row-major), b1, W2 (128x128), b2, W3, b3,
// w4 (128), b4. Gradients are reduced in a fixed order, so training is
// deterministic for a given data order.
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <vector>

#include "kpz.h"
#include "kpz_internal.h"

namespace kpz {
namespace mlp {

constexpr int kW = 128, kIn = 4, kRowsPerBlock = 32;
constexpr int oW1 = 0, oB1 = oW1 + kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + kW * kW, oW3 = oB2 + kW,
              oB3 = oW3 + kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW, kParams = oB4 + 1;
static_assert(kParams == 33793, "parameter count");
constexpr int kPart = kParams + 1;   // per-tile gradient partial + squared-error sum

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float bf(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// One dense layer for a tile of kRowsPerBlock samples: thread j computes unit j,
// z[s] = b[j] + sum_k W[j][k] h[s][k] (h in shared memory, row stride kW).
__device__ __forceinline__ void dense(const __nv_bfloat16* W, const __nv_bfloat16* b, const float (*h)[kW],
                                      int j, float (&z)[kRowsPerBlock]) {
  const float bj = bf(b, j);
#pragma unroll
  for (int s = 0; s < kRowsPerBlock; ++s) z[s] = bj;
  const __nv_bfloat16* row = W + j * kW;
#pragma unroll 1
  for (int k0 = 0; k0 < kW; k0 += 8) {
    float w[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) w[kk] = bf(row, k0 + kk);
#pragma unroll
    for (int s = 0; s < kRowsPerBlock; ++s) {
      const float4 a = *reinterpret_cast<const float4*>(&h[s][k0]);
      const float4 c = *reinterpret_cast<const float4*>(&h[s][k0 + 4]);
      z[s] += w[0] * a.x + w[1] * a.y + w[2] * a.z + w[3] * a.w + w[4] * c.x + w[5] * c.y + w[6] * c.z +
              w[7] * c.w;
    }
  }
}

// Forward pass of a tile: y (and, for training, the pre-activations z1..z3).
__global__ void __launch_bounds__(kW) fwd_kernel(const __nv_bfloat16* __restrict__ P, const float* __restrict__ x,
                                                 int n, float* __restrict__ y, float* __restrict__ zsave) {
  __shared__ __align__(16) float hA[kRowsPerBlock][kW];
  __shared__ __align__(16) float hB[kRowsPerBlock][kW];
  __shared__ float xs[kRowsPerBlock][kIn];
  __shared__ float part[kW / 32][kRowsPerBlock];
  const int j = threadIdx.x, s0 = blockIdx.x * kRowsPerBlock;
  for (int e = j; e < kRowsPerBlock * kIn; e += kW) {
    const int s = e / kIn, c = e % kIn;
    xs[s][c] = (s0 + s < n) ? x[(size_t)(s0 + s) * kIn + c] : 0.f;
  }
  __syncthreads();
  float z[kRowsPerBlock];
  {
    float w[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) w[c] = bf(P + oW1, j * kIn + c);
    const float bj = bf(P + oB1, j);
#pragma unroll
    for (int s = 0; s < kRowsPerBlock; ++s) {
      float a = bj;
#pragma unroll
      for (int c = 0; c < kIn; ++c) a += w[c] * xs[s][c];
      z[s] = a;
    }
  }
  auto store = [&](int layer, float (*h)[kW]) {
#pragma unroll
    for (int s = 0; s < kRowsPerBlock; ++s) {
      if (zsave && s0 + s < n) zsave[((size_t)(s0 + s) * 3 + layer) * kW + j] = z[s];
      h[s][j] = gelu(z[s]);
    }
  };
  store(0, hA);
  __syncthreads();
  dense(P + oW2, P + oB2, hA, j, z);
  store(1, hB);
  __syncthreads();
  dense(P + oW3, P + oB3, hB, j, z);
  const float w4 = bf(P + oW4, j);
#pragma unroll
  for (int s = 0; s < kRowsPerBlock; ++s) {
    if (zsave && s0 + s < n) zsave[((size_t)(s0 + s) * 3 + 2) * kW + j] = z[s];
    float v = w4 * gelu(z[s]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((j & 31) == 0) part[j >> 5][s] = v;
  }
  __syncthreads();
  if (j < kRowsPerBlock && s0 + j < n) {
    float v = bf(P + oB4, 0);
#pragma unroll
    for (int q = 0; q < kW / 32; ++q) v += part[q][j];
    y[s0 + j] = v;
  }
}

// Backward pass of a tile: d(mean squared error)/d(parameters) restricted to
// the tile's samples, written to its own slot of gpart (no atomics).
__global__ void __launch_bounds__(kW) bwd_kernel(const __nv_bfloat16* __restrict__ P, const float* __restrict__ x,
                                                 const float* __restrict__ t, const float* __restrict__ y,
                                                 const float* __restrict__ zsave, int n, float inv_n,
                                                 float* __restrict__ gpart) {
  extern __shared__ __align__(16) float sm[];
  float (*hprev)[kW] = reinterpret_cast<float (*)[kW]>(sm);              // input of the layer
  float (*dz)[kW] = reinterpret_cast<float (*)[kW]>(sm + kRowsPerBlock * kW);     // gradient at its output
  float (*zl)[kW] = reinterpret_cast<float (*)[kW]>(sm + 2 * kRowsPerBlock * kW); // its pre-activation
  float* dy = sm + 3 * kRowsPerBlock * kW;                                        // kRowsPerBlock
  float* xs = dy + kRowsPerBlock;                                                 // kRowsPerBlock * kIn
  const int j = threadIdx.x, s0 = blockIdx.x * kRowsPerBlock;
  float* g = gpart + (size_t)blockIdx.x * kPart;
  for (int e = j; e < kRowsPerBlock * kIn; e += kW) {
    const int s = e / kIn;
    xs[e] = (s0 + s < n) ? x[(size_t)(s0 + s) * kIn + e % kIn] : 0.f;
  }
  if (j < kRowsPerBlock) {
    const float r = (s0 + j < n) ? (y[s0 + j] - t[s0 + j]) : 0.f;
    dy[j] = 2.f * r * inv_n;
    float sq = r * r;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, d);
    if (j == 0) g[kParams] = sq;
  }
  auto zval = [&](int s, int layer, int u) -> float {
    return (s0 + s < n) ? zsave[((size_t)(s0 + s) * 3 + layer) * kW + u] : 0.f;
  };
  // Output layer: dz3 = dy * w4 * gelu'(z3); grads of w4, b4.
  for (int s = 0; s < kRowsPerBlock; ++s) {
    zl[s][j] = zval(s, 2, j);
    hprev[s][j] = gelu(zval(s, 1, j));
  }
  __syncthreads();
  {
    const float w4 = bf(P + oW4, j);
    float gw4 = 0.f;
    for (int s = 0; s < kRowsPerBlock; ++s) {
      gw4 += dy[s] * gelu(zl[s][j]);
      dz[s][j] = dy[s] * w4 * gelu_grad(zl[s][j]);
    }
    g[oW4 + j] = gw4;
    if (j == 0) {
      float gb = 0.f;
      for (int s = 0; s < kRowsPerBlock; ++s) gb += dy[s];
      g[oB4] = gb;
    }
  }
  __syncthreads();
  // Hidden layers 3 and 2: grads of W, b; then the gradient at the input.
  const int oW[2] = {oW3, oW2}, oB[2] = {oB3, oB2};
#pragma unroll 1
  for (int L = 0; L < 2; ++L) {
    // dW[j][k] = sum_s dz[s][j] hprev[s][k]; db[j] = sum_s dz[s][j]
    float db = 0.f;
    for (int s = 0; s < kRowsPerBlock; ++s) db += dz[s][j];
    g[oB[L] + j] = db;
#pragma unroll 1
    for (int k0 = 0; k0 < kW; k0 += 8) {
      float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int s = 0; s < kRowsPerBlock; ++s) {
        const float d = dz[s][j];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) a[kk] += d * hprev[s][k0 + kk];
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) g[oW[L] + j * kW + k0 + kk] = a[kk];
    }
    // gradient at the input of this layer: dh[s][k] = sum_u W[u][k] dz[s][u]  (thread k)
    float dh[kRowsPerBlock];
#pragma unroll
    for (int s = 0; s < kRowsPerBlock; ++s) dh[s] = 0.f;
    const __nv_bfloat16* W = P + oW[L];
#pragma unroll 1
    for (int u = 0; u < kW; ++u) {
      const float w = bf(W, u * kW + j);
#pragma unroll
      for (int s = 0; s < kRowsPerBlock; ++s) dh[s] += w * dz[s][u];
    }
    __syncthreads();   // everyone is done with dz, hprev and zl of this layer
    const int below = 1 - L;   // pre-activation index of the layer whose output we reach
#pragma unroll
    for (int s = 0; s < kRowsPerBlock; ++s) {
      const float zb = zval(s, below, j);
      dz[s][j] = dh[s] * gelu_grad(zb);
      if (L == 0) hprev[s][j] = gelu(zval(s, 0, j));   // input of layer 2 = h1
    }
    __syncthreads();
  }
  // First layer: dW1[j][c] = sum_s dz1[s][j] x[s][c]; db1[j] = sum_s dz1[s][j]
  {
    float a[kIn] = {0.f, 0.f, 0.f, 0.f}, db = 0.f;
    for (int s = 0; s < kRowsPerBlock; ++s) {
      const float d = dz[s][j];
      db += d;
#pragma unroll
      for (int c = 0; c < kIn; ++c) a[c] += d * xs[s * kIn + c];
    }
#pragma unroll
    for (int c = 0; c < kIn; ++c) g[oW1 + j * kIn + c] = a[c];
    g[oB1 + j] = db;
  }
}

// grad[i] = sum over tiles b of gpart[b][i], tiles in order (deterministic).
__global__ void reduce_kernel(const float* __restrict__ gpart, int ntiles, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPart) return;
  float s = 0.f;
  for (int b = 0; b < ntiles; ++b) s += gpart[(size_t)b * kPart + i];
  grad[i] = s;
}

// Adam (Kingma and Ba): master weights in float32, bfloat16 copy for the passes.
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, __nv_bfloat16* __restrict__ P, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  theta[i] = th;
  P[i] = __float2bfloat16_rn(th);
}

__global__ void to_bf16_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kParams) P[i] = __float2bfloat16_rn(theta[i]);
}

constexpr size_t kBwdSmem = (3 * kRowsPerBlock * kW + kRowsPerBlock + kRowsPerBlock * kIn) * sizeof(float);

}  // namespace mlp
}  // namespace kpz

using namespace kpz;
using namespace kpz::mlp;

struct kpz_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* theta = nullptr;       // master parameters
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;        // kPart (last entry: squared-error sum)
  __nv_bfloat16* P = nullptr;   // bfloat16 copy
  uint64_t step = 0;
  // per-call buffers: data (x, t) for `cap` samples, work (y, z, gpart) for `wcap`
  float *x = nullptr, *t = nullptr, *y = nullptr, *z = nullptr, *gpart = nullptr;
  size_t cap = 0, wcap = 0;
};

namespace {

void mlp_release(kpz_mlp* m) {
  float* ptrs[] = {m->theta, m->m, m->v, m->grad, m->x, m->t, m->y, m->z, m->gpart};
  for (float* p : ptrs) if (p) cudaFree(p);
  if (m->P) cudaFree(m->P);
}

// Data buffers for n samples and work buffers for passes over w samples.
kpz_status ensure(kpz_mlp* m, size_t n, size_t w) {
  if (n > m->cap) {
    if (m->x) cudaFree(m->x);
    if (m->t) cudaFree(m->t);
    m->x = m->t = nullptr;
    m->cap = 0;
    if (cudaMalloc(&m->x, n * kIn * 4) != cudaSuccess || cudaMalloc(&m->t, n * 4) != cudaSuccess) {
      cudaGetLastError();
      return KPZ_ENOMEM;
    }
    m->cap = n;
  }
  if (w > m->wcap) {
    float* bufs[] = {m->y, m->z, m->gpart};
    for (float* p : bufs) if (p) cudaFree(p);
    m->y = m->z = m->gpart = nullptr;
    m->wcap = 0;
    const size_t tiles = (w + kRowsPerBlock - 1) / kRowsPerBlock;
    if (cudaMalloc(&m->y, w * 4) != cudaSuccess || cudaMalloc(&m->z, w * 3 * kW * 4) != cudaSuccess ||
        cudaMalloc(&m->gpart, tiles * kPart * 4) != cudaSuccess) {
      cudaGetLastError();
      return KPZ_ENOMEM;
    }
    m->wcap = w;
  }
  return KPZ_OK;
}

// Gradient of the mean squared error over samples [0, n) of the uploaded
// data into m->grad; y and z are filled on the way.
cudaError_t grad_pass(kpz_mlp* m, const float* x, const float* t, int n) {
  const int tiles = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  fwd_kernel<<<tiles, kW, 0, m->stream>>>(m->P, x, n, m->y, m->z);
  count_launch();
  bwd_kernel<<<tiles, kW, kBwdSmem, m->stream>>>(m->P, x, t, m->y, m->z, n, 1.f / (float)n, m->gpart);
  count_launch();
  reduce_kernel<<<(kPart + 255) / 256, 256, 0, m->stream>>>(m->gpart, tiles, m->grad);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

extern "C" {

kpz_status kpz_mlp_create(kpz_mlp** out, const float* params, void* stream) {
  if (!out || !params) return KPZ_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return KPZ_ENODEV;
  kpz_mlp* m = new (std::nothrow) kpz_mlp();
  if (!m) return KPZ_ENOMEM;
  cudaGetDevice(&m->device);
  m->stream = (cudaStream_t)stream;
  if (cudaMalloc(&m->theta, kParams * 4) != cudaSuccess || cudaMalloc(&m->m, kParams * 4) != cudaSuccess ||
      cudaMalloc(&m->v, kParams * 4) != cudaSuccess || cudaMalloc(&m->grad, kPart * 4) != cudaSuccess ||
      cudaMalloc(&m->P, kParams * 2) != cudaSuccess) {
    cudaGetLastError();
    mlp_release(m);
    delete m;
    return KPZ_ENOMEM;
  }
  if (cudaFuncSetAttribute(bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) != cudaSuccess ||
      cudaMemcpyAsync(m->theta, params, kParams * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->m, 0, kParams * 4, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->v, 0, kParams * 4, m->stream) != cudaSuccess) {
    mlp_release(m);
    delete m;
    return KPZ_ECUDA;
  }
  to_bf16_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->theta, m->P);
  count_launch();
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    mlp_release(m);
    delete m;
    return KPZ_ECUDA;
  }
  *out = m;
  return KPZ_OK;
}

kpz_status kpz_mlp_params(kpz_mlp* m, float* params) {
  if (!m || !params) return KPZ_EINVAL;
  if (cudaMemcpyAsync(params, m->theta, kParams * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  return KPZ_OK;
}

kpz_status kpz_mlp_predict(kpz_mlp* m, const float* x, uint32_t n, float* y) {
  if (!m || !x || !y) return KPZ_EINVAL;
  if (n == 0) return KPZ_OK;
  kpz_status st = ensure(m, n, n);
  if (st) return st;
  const int tiles = (int)((n + kRowsPerBlock - 1) / kRowsPerBlock);
  if (cudaMemcpyAsync(m->x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  fwd_kernel<<<tiles, kW, 0, m->stream>>>(m->P, m->x, (int)n, m->y, nullptr);
  count_launch();
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(y, m->y, (size_t)n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  return KPZ_OK;
}

kpz_status kpz_mlp_loss_grad(kpz_mlp* m, const float* x, const float* t, uint32_t n, float* loss, float* grad) {
  if (!m || !x || !t || n == 0) return KPZ_EINVAL;
  kpz_status st = ensure(m, n, n);
  if (st) return st;
  if (cudaMemcpyAsync(m->x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemcpyAsync(m->t, t, (size_t)n * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      grad_pass(m, m->x, m->t, (int)n) != cudaSuccess)
    return KPZ_ECUDA;
  std::vector<float> h(kPart);
  if (cudaMemcpyAsync(h.data(), m->grad, kPart * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  if (grad) for (int i = 0; i < kParams; ++i) grad[i] = h[i];
  if (loss) *loss = h[kParams] / (float)n;
  return KPZ_OK;
}

kpz_status kpz_mlp_train(kpz_mlp* m, const float* x, const float* t, uint32_t n, const uint32_t* order,
                         uint32_t steps, uint32_t batch, float lr, float* last_loss) {
  if (!m || !x || !t || !order || n == 0 || batch == 0 || !(lr > 0.f)) return KPZ_EINVAL;
  // Upload the minibatches already gathered in the order the caller chose:
  // step s uses samples order[s*batch .. s*batch + batch - 1] (indices < n).
  const size_t total = (size_t)steps * batch;
  for (size_t i = 0; i < total; ++i) if (order[i] >= n) return KPZ_EINVAL;
  kpz_status st = ensure(m, total, batch);
  if (st) return st;
  std::vector<float> xg(total * kIn), tg(total);
  for (size_t i = 0; i < total; ++i) {
    for (int c = 0; c < kIn; ++c) xg[i * kIn + c] = x[(size_t)order[i] * kIn + c];
    tg[i] = t[order[i]];
  }
  if (cudaMemcpyAsync(m->x, xg.data(), total * kIn * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemcpyAsync(m->t, tg.data(), total * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (uint32_t s = 0; s < steps; ++s) {
    ++m->step;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    if (grad_pass(m, m->x + (size_t)s * batch * kIn, m->t + (size_t)s * batch, (int)batch) != cudaSuccess)
      return KPZ_ECUDA;
    adam_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->theta, m->m, m->v, m->grad, m->P, lr, b1, b2,
                                                             c1, c2, eps);
    count_launch();
  }
  float sq = 0.f;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&sq, m->grad + kParams, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  if (last_loss) *last_loss = sq / (float)batch;
  return KPZ_OK;
}

void kpz_mlp_free(kpz_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  mlp_release(m);
  delete m;
}

}  // extern "C"
