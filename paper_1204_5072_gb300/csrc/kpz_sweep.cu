// kpz_sweep.cu -- one Monte Carlo sweep of the octahedron KPZ model on GB300.
//
// One launch = one sweep. The resident warps take runs of P.run tiles of one
// tile row from a work queue (run::sweep_run, kpz_run.cuh); the Sec. 3
// decomposition and the Sec. 2.1 update rule are documented there and in
// kpz_rounds.cuh. On the p = 1, q = 0 path the Philox round keys are read from
// shared memory instead of being advanced per draw.
#include <algorithm>
#include <mutex>

#include "kpz_run.cuh"

namespace kpz {
namespace {

using run::WarpStage;
using run::kFull;
using run::kMaxWarpsPerCta;

// Persistent sweep: the resident warps take chunks of P.run tiles of one
// tile row from a work queue (row-major order, one atomic per chunk, fetched
// a chunk ahead), so faster SMs take more chunks and the tail is one chunk.
// Every warp makes exactly one fetch past the last chunk; the warp whose
// fetch is the last of all (nchunks + W - 1) returns the counter to zero for
// the next launch.
template <bool kGeneral, int CR, bool kC2>
__global__ void __launch_bounds__(256, CR == 1 ? (kGeneral ? 2 : 3) : (kGeneral ? 1 : 2))
sweep_kernel(const SweepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpStage<CR>& ws = reinterpret_cast<WarpStage<CR>*>(smem_raw)[threadIdx.x >> 5];
  __shared__ uint4 rk[kPhiloxRounds / 2];   // Philox round keys of (k0, k1)
  if (!kGeneral && threadIdx.x < kPhiloxRounds / 2) {
    const uint32_t r = 2u * threadIdx.x;
    rk[threadIdx.x] = make_uint4(P.k0 + r * kPhiloxWeylA, P.k1 + r * kPhiloxWeylB,
                                 P.k0 + (r + 1u) * kPhiloxWeylA, P.k1 + (r + 1u) * kPhiloxWeylB);
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  const uint32_t cpr = P.ntx / P.run;              // chunks per tile row
  const uint32_t nchunks = cpr * P.nty;
  const uint32_t L = P.g.L;
  const uint32_t s = (uint32_t)(*P.t_dev) + P.s_add;
  // Device layer: random origin of this sweep's tile grid.
  const uint4 o = philox(kTagOrigin << 28, 0u, s, P.sample, P.k0, P.k1);
  const uint32_t ox = o.x & (L - 1u), oy = o.y & (L - 1u);
  uint32_t c = 0;
  if (lane == 0) c = atomicAdd(P.queue, 1u);
  c = __shfl_sync(kFull, c, 0);
  while (c < nchunks) {
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(P.queue, 1u);
    const uint32_t ty = c / cpr;
    run::sweep_run<kGeneral, CR, !kGeneral, false, kC2>(P, ws, rk, lane, s, ox, oy, ty, (c - ty * cpr) * P.run,
                                                       P.run);
    c = __shfl_sync(kFull, next, 0);
  }
  if (lane == 0 && c == nchunks + W - 1u) atomicExch(P.queue, 0u);
}

// Resident CTAs per SM of one sweep kernel at wpc warps per CTA (cached per device).
template <bool kGeneral, int CR, bool kC2>
cudaError_t resident_ctas(uint32_t wpc, uint32_t& ctas) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static uint32_t cache[kMaxDev][kMaxWarpsPerCta + 1] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < kMaxDev && cache[dev][wpc]) { ctas = cache[dev][wpc]; return cudaSuccess; }
  const int bytes = (int)(kMaxWarpsPerCta * sizeof(WarpStage<CR>));
  e = cudaFuncSetAttribute(sweep_kernel<kGeneral, CR, kC2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<kGeneral, CR, kC2>, (int)(wpc * 32u),
                                                    wpc * sizeof(WarpStage<CR>));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  ctas = (uint32_t)(per_sm > 0 ? per_sm : 1) * (uint32_t)(sms > 0 ? sms : 1);
  if (dev < kMaxDev) cache[dev][wpc] = ctas;
  return cudaSuccess;
}

template <bool kGeneral, int CR, bool kC2 = false>
cudaError_t launch_cr(const SweepParams& P, uint32_t wpc, cudaStream_t st) {
  uint32_t ctas = 0;
  cudaError_t e = resident_ctas<kGeneral, CR, kC2>(wpc, ctas);
  if (e != cudaSuccess) return e;
  // One wave of resident warps, fewer if there are fewer tiles than warps.
  const uint64_t tiles = (uint64_t)P.ntx * P.nty;
  const uint64_t blocks = std::min<uint64_t>(ctas, (tiles + wpc - 1) / wpc);
  sweep_kernel<kGeneral, CR, kC2><<<(unsigned)blocks, wpc * 32u, wpc * sizeof(WarpStage<CR>), st>>>(P);
  return cudaSuccess;
}

__global__ void advance_kernel(uint64_t* t_dev, uint32_t n) { *t_dev += n; }

}  // namespace

cudaError_t launch_sweep(const SweepParams& P, uint32_t warps_per_cta, cudaStream_t st) {
  // The tile height 128 CR follows from the number of tile rows.
  const uint32_t wpc = warps_per_cta ? warps_per_cta : 8u;
  if (wpc > kMaxWarpsPerCta) return cudaErrorInvalidValue;
  const uint32_t tile_y = P.g.L / P.nty;
  cudaError_t e;
  const bool general = !(P.Tp == 65536u && P.Tq == 0u);
  if (P.cell == 2u && tile_y == kTile)
    e = general ? launch_cr<true, 1, true>(P, wpc, st) : launch_cr<false, 1, true>(P, wpc, st);
  else if (P.cell == 2u)
    return cudaErrorInvalidValue;
  else if (tile_y == kTile)
    e = general ? launch_cr<true, 1>(P, wpc, st) : launch_cr<false, 1>(P, wpc, st);
  else if (tile_y == 2u * kTile)
    e = general ? launch_cr<true, 2>(P, wpc, st) : launch_cr<false, 2>(P, wpc, st);
  else
    return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_advance(uint64_t* t_dev, uint32_t n, cudaStream_t st) {
  advance_kernel<<<1, 1, 0, st>>>(t_dev, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kpz
