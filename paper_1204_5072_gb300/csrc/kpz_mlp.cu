// kpz_mlp.cu -- the learned surrogate: a 4-128-128-128-1 GELU MLP with
// bfloat16 weights and float32 arithmetic, trained with Adam by the kernels
// below (forward and backward on the tcgen05 tensor cores, gradient
// reduction, update).
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

constexpr int kW = 128, kIn = 4;
constexpr int oW1 = 0, oB1 = oW1 + kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + kW * kW, oW3 = oB2 + kW,
              oB3 = oW3 + kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW, kParams = oB4 + 1;
static_assert(kParams == 33793, "parameter count");
constexpr int kPart = kParams + 1;   // per-tile gradient partial + squared-error sum

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float bf(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// ---------------------------------------------------------------------------
// The 128 x 128 layers on the 5th-generation tensor cores (tcgen05). A tile
// is 128 samples, four threads per sample (each a quarter of the units). In
// the forward pass the two 128 x 128 layers run as
// D[s][j] = sum_k A[s][k] W[j][k] with M = N = K = 128: A (activations) and W
// (weights) in shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices, 128 B apart along K, 2048 B apart along the
// rows), the float32 accumulator in tensor memory (lane = sample, column =
// unit). The MMA takes bfloat16 operands; the weights are bfloat16 already,
// each float32 activation a is split into hi = bf16(a) and lo = bf16(a - hi),
// and two chains of MMAs (hi, then lo, 8 of K = 16 each) accumulate
// sum_k (hi + lo) W, which agrees with the float32 product to about 2^-16
// relative. One thread issues the MMAs and commits them to an mbarrier; every
// wait on it is bounded in time (a timeout sets *err and the host reports it).
namespace tc {

constexpr int kM = 128;                              // samples per tile (MMA M)
constexpr int kQ = 4;                                // threads per sample: a quarter of the units each
constexpr int kThreads = kM * kQ;                    // 16 warps; warp w reads tensor-memory lanes 32 (w % 4)
constexpr uint32_t kOpBytes = (uint32_t)kW * kW * 2;  // one 128 x 128 bfloat16 operand
constexpr size_t kSmem = 3 * (size_t)kOpBytes;       // A hi, A lo, W
// Instruction descriptor of tcgen05.mma kind::f16: float32 accumulator
// (bits 4-5 = 1), bfloat16 A and B (bits 7-9, 10-12 = 1), both K-major,
// N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kW >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);
constexpr uint64_t kWaitNs = 1000000000ull;          // bound of every wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) of a 128 x 128 bfloat16 operand.
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 16 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K: 128), stride byte offset (between
// 8-row groups: 2048), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(2048u >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// D (tensor memory) = (Ahi + Alo) W^T over K = 128, then commit to mbar.
__device__ __forceinline__ void mma_chain(uint32_t taddr, uint32_t ahi, uint32_t alo, uint32_t b, uint32_t mbar) {
#pragma unroll
  for (int part = 0; part < 2; ++part) {
#pragma unroll
    for (int kk = 0; kk < kW / 16; ++kk) {
      const uint64_t ad = sdesc((part ? alo : ahi) + kk * 256u);
      const uint64_t bd = sdesc(b + kk * 256u);
      const uint32_t acc = (part | kk) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
          "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Wait until phase `parity` of the mbarrier has completed; false on timeout.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}

// 32 consecutive float32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void ld32(uint32_t ta, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Eight activations h[0..7] of units j0..j0+7 (j0 % 8 == 0) of sample row s,
// split into bfloat16 hi and lo parts, as one 16-byte core-matrix row each.
__device__ __forceinline__ void put8(unsigned char* Ahi, unsigned char* Alo, int s, int j0, const float* h) {
  __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hi[i] = __float2bfloat16_rn(h[i]);
    lo[i] = __float2bfloat16_rn(h[i] - __bfloat162float(hi[i]));
  }
  *reinterpret_cast<uint4*>(Ahi + cm_off(s, j0)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(Alo + cm_off(s, j0)) = *reinterpret_cast<const uint4*>(lo);
}

// W (128 x 128 bfloat16, row = output unit, K contiguous) into the operand layout.
__device__ __forceinline__ void stage_w(unsigned char* Bs, const __nv_bfloat16* W, int t) {
#pragma unroll 4
  for (int q = t; q < kW * kW / 8; q += kThreads) {
    const int row = q >> 4, k0 = (q & 15) * 8;
    *reinterpret_cast<uint4*>(Bs + cm_off(row, k0)) = *reinterpret_cast<const uint4*>(W + row * kW + k0);
  }
}

__device__ __forceinline__ void fence_to_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace tc

// Forward pass of a tile of 128 samples: y (and, for training, the
// pre-activations z1..z3 in zsave). Thread (sample s, quarter q) handles units
// 32 q .. 32 q + 31 of sample s; warps 4 q .. 4 q + 3 read columns 32 q ..
// 32 q + 31 of the tensor-memory lanes of their samples.
__global__ void __launch_bounds__(tc::kThreads, 1) fwd_kernel(const __nv_bfloat16* __restrict__ P,
                                                              const float* __restrict__ x, int n,
                                                              float* __restrict__ y, float* __restrict__ zsave,
                                                              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* Ahi = smem_tc;
  unsigned char* Alo = smem_tc + tc::kOpBytes;
  unsigned char* Bs = smem_tc + 2 * tc::kOpBytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ float part[tc::kQ][tc::kM];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int s = (warp & 3) * 32 + (tid & 31), q = warp >> 2, u0 = 32 * q;
  const int gs = blockIdx.x * tc::kM + s;
  const bool live = gs < n;
  float xin[kIn];
#pragma unroll
  for (int c = 0; c < kIn; ++c) xin[c] = live ? x[(size_t)gs * kIn + c] : 0.f;
  // Layer 1 (K = 4) on the CUDA cores, straight into the operand A.
#pragma unroll 1
  for (int j0 = u0; j0 < u0 + 32; j0 += 8) {
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = j0 + i;
      float z = bf(P + oB1, j);
#pragma unroll
      for (int c = 0; c < kIn; ++c) z += bf(P + oW1, j * kIn + c) * xin[c];
      if (zsave && live) zsave[((size_t)gs * 3 + 0) * kW + j] = z;
      h[i] = gelu(z);
    }
    tc::put8(Ahi, Alo, s, j0, h);
  }
  tc::stage_w(Bs, P + oW2, tid);
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tc::smem_u32(&taddr_s)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_to_mma();
  const uint32_t taddr = taddr_s, lanes = taddr + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t mb = tc::smem_u32(&mbar);
  bool ok = true;
  const int oBl[2] = {oB2, oB3};
  float out = 0.f;
#pragma unroll 1
  for (int layer = 0; layer < 2; ++layer) {
    if (tid == 0) tc::mma_chain(taddr, tc::smem_u32(Ahi), tc::smem_u32(Alo), tc::smem_u32(Bs), mb);
    ok = tc::wait_phase(mb, (uint32_t)layer) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float v[32];
    tc::ld32(lanes + (uint32_t)u0, v);
#pragma unroll
    for (int g = 0; g < 32; g += 8) {
      float h[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = u0 + g + i;
        const float z = v[g + i] + bf(P + oBl[layer], j);
        if (zsave && live) zsave[((size_t)gs * 3 + 1 + layer) * kW + j] = z;
        h[i] = gelu(z);
        if (layer == 1) out += bf(P + oW4, j) * h[i];
      }
      if (layer == 0) tc::put8(Ahi, Alo, s, u0 + g, h);
    }
    if (layer == 0) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();   // every lane read layer 2 and the MMAs are done with W2: restage
      tc::stage_w(Bs, P + oW3, tid);
      tc::fence_to_mma();
    }
  }
  part[q][s] = out;
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (q == 0 && live) y[gs] = ((part[0][s] + part[1][s]) + part[2][s]) + part[3][s] + bf(P + oB4, 0);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(taddr));
}

namespace tc {

// D (tensor memory) = sum over the npair operand pairs (a[i], b[i]) of
// a[i] b[i]^T, K = 128 each, then commit to mbar.
__device__ __forceinline__ void mma_pairs(uint32_t taddr, const uint32_t* a, const uint32_t* b, int npair,
                                          uint32_t mbar) {
#pragma unroll 1
  for (int pr = 0; pr < npair; ++pr) {
#pragma unroll
    for (int kk = 0; kk < kW / 16; ++kk) {
      const uint64_t ad = sdesc(a[pr] + kk * 256u);
      const uint64_t bd = sdesc(b[pr] + kk * 256u);
      const uint32_t acc = (pr | kk) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
          "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Element (row, k) of a pair of operands as bfloat16 hi and lo parts.
__device__ __forceinline__ void put1(unsigned char* Xhi, unsigned char* Xlo, int row, int k, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(Xhi + cm_off(row, k)) = hi;
  *reinterpret_cast<__nv_bfloat16*>(Xlo + cm_off(row, k)) = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__device__ __forceinline__ float get1(const unsigned char* Xhi, const unsigned char* Xlo, int row, int k) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(Xhi + cm_off(row, k))) +
         __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(Xlo + cm_off(row, k)));
}

// W^T of a 128 x 128 bfloat16 weight matrix (row = output unit) into the
// operand layout: element (k, u) = W[u][k].
__device__ __forceinline__ void stage_wt(unsigned char* Bs, const __nv_bfloat16* W, int t) {
#pragma unroll 2
  for (int q = t; q < kW * kW / 8; q += kThreads) {
    const int k = q & (kW - 1), u0 = (q >> 7) * 8;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = W[(u0 + i) * kW + k];
    *reinterpret_cast<uint4*>(Bs + cm_off(k, u0)) = *reinterpret_cast<const uint4*>(v);
  }
}

}  // namespace tc

// Backward pass of a tile of 128 samples: d(mean squared error)/d(parameters)
// restricted to the tile's samples, written to its own slot of gpart (no
// atomics). Per hidden layer (3, then 2) two tensor-core products: the weight
// gradient dW[u][k] = sum_s dz[s][u] h[s][k] (M = units, K = samples; dz and h
// split into bfloat16 hi and lo, three MMA chains hi.hi + hi.lo + lo.hi, in
// tensor-memory columns 128..255) and the gradient at the layer's input
// dh[s][k] = sum_u dz[s][u] W[u][k] (M = samples, K = units; two chains, in
// columns 0..127). Thread (sample s, quarter q) handles units 32 q .. 32 q + 31
// of sample s. Column sums over the samples (biases, the output and the first
// layer) are taken per unit in four quarters of 32 samples, added in a fixed
// order, so a call is deterministic.
__global__ void __launch_bounds__(tc::kThreads, 1) bwd_kernel(const __nv_bfloat16* __restrict__ P,
                                                              const float* __restrict__ x, const float* __restrict__ t,
                                                              const float* __restrict__ y,
                                                              const float* __restrict__ zsave, int n, float inv_n,
                                                              float* __restrict__ gpart, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* X0 = smem_tc;                       // operand buffers, 32 KB each
  unsigned char* X1 = smem_tc + tc::kOpBytes;
  unsigned char* X2 = smem_tc + 2 * tc::kOpBytes;
  unsigned char* X3 = smem_tc + 3 * tc::kOpBytes;
  float* dzT = reinterpret_cast<float*>(smem_tc);    // layer 1: dz1 as [unit][sample] float32 (X0, X1)
  __shared__ float dy[tc::kM];
  __shared__ float xs[tc::kM * kIn];
  __shared__ float sq_part[4];
  __shared__ float red[tc::kQ][tc::kM][kIn + 1];     // per-quarter column sums
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int s = (warp & 3) * 32 + (tid & 31), q = warp >> 2, u0 = 32 * q;   // sample role
  const int uu = tid & (tc::kM - 1), qq = tid >> 7, k0 = 32 * qq;            // unit role: unit uu, samples k0..k0+31
  const int s0 = blockIdx.x * tc::kM;
  float* g = gpart + (size_t)blockIdx.x * kPart;
  auto zval = [&](int smp, int layer, int u) -> float {   // zero beyond the last sample
    return (s0 + smp < n) ? zsave[((size_t)(s0 + smp) * 3 + layer) * kW + u] : 0.f;
  };
  // Sum of the four quarters' partials of unit uu (fixed order), by the threads of quarter 0.
  auto combine = [&](int c) -> float { return ((red[0][uu][c] + red[1][uu][c]) + red[2][uu][c]) + red[3][uu][c]; };
  if (q == 0) {
    const int gs = s0 + s;
    const bool live = gs < n;
#pragma unroll
    for (int c = 0; c < kIn; ++c) xs[s * kIn + c] = live ? x[(size_t)gs * kIn + c] : 0.f;
    const float r = live ? (y[gs] - t[gs]) : 0.f;
    dy[s] = 2.f * r * inv_n;
    float sq = r * r;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, d);
    if ((tid & 31) == 0) sq_part[warp] = sq;
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tc::smem_u32(&taddr_s)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = taddr_s, lanes = taddr + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t mb = tc::smem_u32(&mbar);
  const uint32_t x0 = tc::smem_u32(X0), x1 = tc::smem_u32(X1), x2 = tc::smem_u32(X2), x3 = tc::smem_u32(X3);
  uint32_t phase = 0;
  bool ok = true;
  if (tid == 0) g[kParams] = ((sq_part[0] + sq_part[1]) + sq_part[2]) + sq_part[3];
  // Output layer: grads of w4 and b4.
  {
    float gw4 = 0.f, gb = 0.f;
#pragma unroll
    for (int k = k0; k < k0 + 32; ++k) {
      gw4 += dy[k] * gelu(zval(k, 2, uu));
      gb += dy[k];
    }
    red[qq][uu][0] = gw4;
    red[qq][uu][1] = gb;
  }
  __syncthreads();
  if (qq == 0) {
    g[oW4 + uu] = combine(0);
    if (uu == 0) g[oB4] = combine(1);
  }
  __syncthreads();
  const int oW[2] = {oW3, oW2}, oB[2] = {oB3, oB2};
#pragma unroll 1
  for (int L = 0; L < 2; ++L) {
    const int zl = 2 - L;   // pre-activation of this layer's output: z3, then z2
    // dz (sample s, units u0..u0+31) -> X0/X1 transposed (row = unit), h at the
    // layer's input -> X2/X3 transposed. Layer 3: dz3 = dy w4 gelu'(z3); layer 2:
    // dz2 = dh2 gelu'(z2), dh2 from tensor memory.
    {
      float dh[32];
      if (L == 1) tc::ld32(lanes + (uint32_t)u0, dh);
#pragma unroll 16
      for (int i = 0; i < 32; ++i) {
        const int u = u0 + i;
        const float d = (L == 0) ? dy[s] * bf(P + oW4, u) : dh[i];
        tc::put1(X0, X1, u, s, d * gelu_grad(zval(s, zl, u)));
        tc::put1(X2, X3, u, s, gelu(zval(s, zl - 1, u)));
      }
    }
    tc::fence_to_mma();
    // Bias gradient: column sum of dz over the samples.
    {
      float db = 0.f;
#pragma unroll 8
      for (int k = k0; k < k0 + 32; ++k) db += tc::get1(X0, X1, uu, k);
      red[qq][uu][0] = db;
    }
    __syncthreads();   // every column read before X0/X1 are rewritten below
    if (qq == 0) g[oB[L] + uu] = combine(0);
    // dW[u][k] into columns 128..255.
    if (tid == 0) {
      const uint32_t a[3] = {x0, x0, x1}, b[3] = {x2, x3, x2};
      tc::mma_pairs(taddr + 128u, a, b, 3, mb);
    }
    ok = tc::wait_phase(mb, phase) && ok;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      float v[32];
      tc::ld32(lanes + 128u + (uint32_t)u0, v);    // row = unit s, columns u0..u0+31
      float* dst = g + oW[L] + s * kW + u0;        // a tile's slot is not 16-byte aligned: scalar stores
#pragma unroll
      for (int i = 0; i < 32; ++i) dst[i] = v[i];
    }
    // dz again, now as rows (sample s) in X0/X1; W^T in X2.
    {
      float dh[32];
      if (L == 1) tc::ld32(lanes + (uint32_t)u0, dh);
#pragma unroll
      for (int g8 = 0; g8 < 32; g8 += 8) {
        float d8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int u = u0 + g8 + i;
          const float d = (L == 0) ? dy[s] * bf(P + oW4, u) : dh[g8 + i];
          d8[i] = d * gelu_grad(zval(s, zl, u));
        }
        tc::put8(X0, X1, s, u0 + g8, d8);
      }
    }
    tc::stage_wt(X2, P + oW[L], tid);
    tc::fence_to_mma();
    // dh at the layer's input into columns 0..127.
    if (tid == 0) {
      const uint32_t a[2] = {x0, x1}, b[2] = {x2, x2};
      tc::mma_pairs(taddr, a, b, 2, mb);
    }
    ok = tc::wait_phase(mb, phase) && ok;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // First layer: dz1 = dh1 gelu'(z1) into dzT[u][s], then per unit
  // dW1[u][c] = sum_s dz1 x[s][c], db1[u] = sum_s dz1.
  {
    float dh[32];
    tc::ld32(lanes + (uint32_t)u0, dh);
#pragma unroll
    for (int i = 0; i < 32; ++i) dzT[(u0 + i) * tc::kM + s] = dh[i] * gelu_grad(zval(s, 0, u0 + i));
  }
  __syncthreads();
  {
    float a[kIn] = {0.f, 0.f, 0.f, 0.f}, db = 0.f;
#pragma unroll 8
    for (int k = k0; k < k0 + 32; ++k) {
      const float d = dzT[uu * tc::kM + k];
      db += d;
#pragma unroll
      for (int c = 0; c < kIn; ++c) a[c] += d * xs[k * kIn + c];
    }
#pragma unroll
    for (int c = 0; c < kIn; ++c) red[qq][uu][c] = a[c];
    red[qq][uu][kIn] = db;
  }
  __syncthreads();
  if (qq == 0) {
#pragma unroll
    for (int c = 0; c < kIn; ++c) g[oW1 + uu * kIn + c] = combine(c);
    g[oB1 + uu] = combine(kIn);
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(taddr));
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

constexpr size_t kBwdSmem = 4 * (size_t)tc::kOpBytes;   // four tensor-core operand buffers

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
  int* err = nullptr;           // set by the forward kernel when a tensor-core wait timed out
};

namespace {

void mlp_release(kpz_mlp* m) {
  float* ptrs[] = {m->theta, m->m, m->v, m->grad, m->x, m->t, m->y, m->z, m->gpart};
  for (float* p : ptrs) if (p) cudaFree(p);
  if (m->P) cudaFree(m->P);
  if (m->err) cudaFree(m->err);
}

// KPZ_OK, or KPZ_ETIMEOUT when a forward kernel's tensor-core wait ran out
// (the flag is then cleared); the stream is synchronised.
kpz_status check_err(kpz_mlp* m) {
  int e = 0;
  if (cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  if (e) {
    cudaMemsetAsync(m->err, 0, 4, m->stream);
    return KPZ_ETIMEOUT;
  }
  return KPZ_OK;
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
    const size_t tiles = (w + tc::kM - 1) / tc::kM;
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
  const int tiles = (n + tc::kM - 1) / tc::kM;
  fwd_kernel<<<tiles, tc::kThreads, tc::kSmem, m->stream>>>(m->P, x, n, m->y, m->z, m->err);
  count_launch();
  bwd_kernel<<<tiles, tc::kThreads, kBwdSmem, m->stream>>>(m->P, x, t, m->y, m->z, n, 1.f / (float)n, m->gpart,
                                                      m->err);
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
      cudaMalloc(&m->P, kParams * 2) != cudaSuccess || cudaMalloc(&m->err, 4) != cudaSuccess) {
    cudaGetLastError();
    mlp_release(m);
    delete m;
    return KPZ_ENOMEM;
  }
  if (cudaFuncSetAttribute(bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) != cudaSuccess ||
      cudaFuncSetAttribute(fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem) != cudaSuccess ||
      cudaMemsetAsync(m->err, 0, 4, m->stream) != cudaSuccess ||
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
  if (cudaMemcpyAsync(m->x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  fwd_kernel<<<(n + tc::kM - 1) / tc::kM, tc::kThreads, tc::kSmem, m->stream>>>(m->P, m->x, (int)n, m->y, nullptr,
                                                                         m->err);
  count_launch();
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(y, m->y, (size_t)n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return KPZ_ECUDA;
  return check_err(m);
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
  return check_err(m);
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
  return check_err(m);
}

void kpz_mlp_free(kpz_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  mlp_release(m);
  delete m;
}

}  // extern "C"
