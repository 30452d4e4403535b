// kpz_peak.cu -- throughput probe of the integer logic (ALU) pipe, the unit
// that bounds the sweep kernel. Not part of the paper's method: it measures
// the denominator of the sweep's roofline on the GPU at hand.
//
// Every thread runs kChains independent chains of three-input XORs (LOP3),
// each step depending on the previous step of its own chain, so the pipe
// sees kChains independent instructions per thread at a time; one full wave
// of resident CTAs keeps every SM sub-partition busy.
#include <cstdint>
#include <cuda_runtime.h>

#include "kpz.h"
#include "kpz_internal.h"

namespace kpz {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
__device__ uint32_t g_peak_sink;

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__global__ void __launch_bounds__(kThreads) alu_probe_kernel(uint32_t iters, uint32_t seed) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (uint32_t)c;
  const uint32_t k0 = seed * 3u + blockIdx.x, k1 = seed * 5u + 7u;
#pragma unroll 1
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = xor3(x[c], (r & 1) ? k0 : k1, x[(c + 1) % kChains]);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= x[c];
  if (acc == 0x12345678u) g_peak_sink = acc;   // keeps the chains live
}

}  // namespace
}  // namespace kpz

extern "C" kpz_status kpz_alu_peak(double* lane_ops_per_s, double* kernel_ms) {
  using namespace kpz;
  if (!lane_ops_per_s) return KPZ_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_probe_kernel, kThreads, 0) != cudaSuccess)
    return KPZ_ECUDA;
  const uint32_t blocks = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
  const uint32_t iters = 4096;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return KPZ_ECUDA;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  alu_probe_kernel<<<blocks, kThreads, 0, st>>>(64, 1u);   // warm-up
  count_launch();
  cudaEventRecord(e0, st);
  alu_probe_kernel<<<blocks, kThreads, 0, st>>>(iters, 2u);
  count_launch();
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (!ok || cudaGetLastError() != cudaSuccess || ms <= 0.f) return KPZ_ECUDA;
  const double ops = (double)blocks * kThreads * iters * 16.0 * kChains;
  *lane_ops_per_s = ops / (ms * 1e-3);
  if (kernel_ms) *kernel_ms = ms;
  return KPZ_OK;
}
