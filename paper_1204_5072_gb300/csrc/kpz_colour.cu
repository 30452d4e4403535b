// kpz_colour.cu -- random-sequential updates by colour classes: a parallel
// reference for the random-sequential dynamics the decomposition approximates
// (the paper checks its decomposed runs against it, Sec. 3.1 and 4).
//
// Sweep s is K = 4 * 2^m sub-steps; sub-step i draws one of the four period-2
// sublattices (class c, sites x = c & 1, y = c >> 1 mod 2) and attempts each of
// its sites with probability 2^-m (rule eq. rule, Sec. 2.1). Sites of one class
// are never neighbours, so the attempts of a sub-step commute and can all run
// at once; with thin subsets (large m) the dynamics approaches one attempt at a
// uniformly random site at a time. One launch per sub-step.
//
// Work layout: 128 x 128 tiles anchored at (0, 0), so a tile's 32 cells of a
// cell row are exactly one lattice word per plane (kpz_common.cuh): the tile
// owns its words and writes them back whole; a warp takes one tile at a time
// (lane = cell row) and reads the sites around the tile (all of other classes,
// constant during the launch) as halos. The random streams (tags 6 and 7) are
// defined in the header of the CPU oracle; both sides implement them.
#include <algorithm>
#include <mutex>

#include "kpz_internal.h"
#include "kpz_rounds.cuh"

namespace kpz {
namespace {

using rounds::kFull;
using rounds::TileCtx;

constexpr uint32_t kWarps = 8;

// Selected moves of the class sites (CA + 2i, CB + 2j) of every storage cell
// of this lane's cell row, then the flips. sel[j][i]: cells attempting that
// site in this sub-step. hxl / hyu: left / upper neighbours of the tile (tc),
// hx / hy: right / lower ones.
template <int CA, int CB, bool kGeneral>
__device__ __forceinline__ void colour_round(uint32_t (&T)[4][4], const uint32_t (&hx)[4],
                                             const uint32_t (&hy)[4], const uint32_t (&sel)[2][2],
                                             const SweepParams& P, const TileCtx& tc, uint32_t lane,
                                             uint32_t i_sub, int kPar, int& dh) {
  uint32_t ysh[2];
  if (CB == 0) {
    ysh[0] = __shfl_up_sync(kFull, T[3][CA], 1);
    ysh[1] = __shfl_up_sync(kFull, T[3][CA + 2], 1);
    if (lane == 0u) { ysh[0] = tc.hyu[CA]; ysh[1] = tc.hyu[CA + 2]; }
  } else {
    const uint32_t d0 = __shfl_down_sync(kFull, T[0][CA], 1);
    const uint32_t d1 = __shfl_down_sync(kFull, T[0][CA + 2], 1);
    ysh[0] = tc.last_lane ? hy[CA] : d0;
    ysh[1] = tc.last_lane ? hy[CA + 2] : d1;
  }
  uint32_t fmin[2][2], fmax[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int xp = CA + 2 * i, yp = CB + 2 * j;
      const uint32_t s = T[yp][xp];
      const uint32_t nL = (xp > 0) ? T[yp][xp > 0 ? xp - 1 : 0] : ((T[yp][3] << 1) | tc.hxl[yp]);
      const uint32_t nR = (xp < 3) ? T[yp][xp < 3 ? xp + 1 : 3] : __funnelshift_r(T[yp][0], hx[yp], 1);
      const uint32_t nU = (yp > 0) ? T[yp > 0 ? yp - 1 : 0][xp] : ysh[i];
      const uint32_t nD = (yp < 3) ? T[yp < 3 ? yp + 1 : 3][xp] : ysh[i];
      const uint32_t v = ((kPar + xp + yp) & 1) ? ~s : s;   // bit of a higher neighbour
      const uint32_t hL = ~(nL ^ v), hR = ~(nR ^ v), hU = ~(nU ^ v), hD = ~(nD ^ v);
      fmin[j][i] = sel[j][i] & hL & hR & hU & hD;
      fmax[j][i] = kGeneral ? (sel[j][i] & ~hL & ~hR & ~hU & ~hD) : 0u;
    }
  if (kGeneral) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        uint32_t AP, AQ;
        rounds::acceptance<false>(P, tc, (kTagClassAcc << 28) | (i_sub << 9) | (lane << 4) |
                                             (uint32_t)((2 * j + i) << 2),
                                  fmin[j][i], fmax[j][i], AP, AQ);
        fmin[j][i] &= AP;
        fmax[j][i] &= AQ;
      }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int xp = CA + 2 * i, yp = CB + 2 * j;
      if (tc.track && lane == 0u && xp == 0 && yp == 0)   // site (0,0): cell 0 of tile 0
        dh += 2 * (int)(fmin[j][i] & 1u) - 2 * (int)(fmax[j][i] & 1u);
      T[yp][xp] ^= fmin[j][i] | fmax[j][i];
    }
}

template <bool kGeneral>
__device__ __forceinline__ void colour_tile(const SweepParams& P, uint32_t lane, uint32_t s,
                                            uint32_t i_sub, uint32_t m, uint32_t cls,
                                            uint32_t tx, uint32_t ty) {
  const uint32_t NR = P.g.NR, NB = P.g.NB;
  const size_t kstride = (size_t)kPlanes * NR;
  const uint32_t R = ty * 32u + lane;                       // storage cell row of this lane
  const uint32_t Ru = (ty * 32u + NR - 1u) & (NR - 1u);     // row above the tile
  const uint32_t Rd = (ty * 32u + 32u) & (NR - 1u);         // row below the tile
  uint32_t* w = P.lat + (size_t)tx * kstride;
  const uint32_t* wl = P.lat + (size_t)((tx + NB - 1u) & (NB - 1u)) * kstride;
  const uint32_t* wr = P.lat + (size_t)((tx + 1u) & (NB - 1u)) * kstride;
  TileCtx tc;
  uint32_t T[4][4], hx[4], hy[4];
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq) {
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq) T[yq][xq] = __ldcg(w + (size_t)plane(yq, xq) * NR + R);
    tc.hxl[yq] = __ldcg(wl + (size_t)plane(yq, 3) * NR + R) >> 31;   // site left of the tile
    hx[yq] = __ldcg(wr + (size_t)plane(yq, 0) * NR + R) & 1u;         // site right of the tile
  }
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    hy[xq] = lane == 31u ? __ldcg(w + (size_t)plane(0, xq) * NR + Rd) : 0u;
    tc.hyu[xq] = lane == 0u ? __ldcg(w + (size_t)plane(3, xq) * NR + Ru) : 0u;
  }
  tc.tid = ty * P.ntx + tx;
  tc.s = s;
  tc.last_lane = lane == 31u;
  tc.track = tx == 0u && ty == 0u && cls == 0u;
  // Cells attempting each class site: 2^-m subsets from tag 6.
  uint32_t sel[2][2];
#pragma unroll
  for (uint32_t a = 0; a < 4; ++a) {
    uint32_t word = ~0u;
    if (m) {
      const uint4 S = philox((kTagClass << 28) | (i_sub << 9) | (lane << 2) | a, tc.tid, s, P.sample, P.k0, P.k1);
      const uint32_t q[4] = {S.x, S.y, S.z, S.w};
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k)
        if (k < m) word &= q[k];
    }
    sel[a >> 1][a & 1u] = word;
  }
  const int par = (int)(P.g.par & 1u);   // parity of the tile's site (0,0): tiles start at even sites
  int dh = 0;
  switch (cls) {
    case 0: colour_round<0, 0, kGeneral>(T, hx, hy, sel, P, tc, lane, i_sub, par, dh); break;
    case 1: colour_round<1, 0, kGeneral>(T, hx, hy, sel, P, tc, lane, i_sub, par, dh); break;
    case 2: colour_round<0, 1, kGeneral>(T, hx, hy, sel, P, tc, lane, i_sub, par, dh); break;
    default: colour_round<1, 1, kGeneral>(T, hx, hy, sel, P, tc, lane, i_sub, par, dh); break;
  }
  if (tc.track && lane == 0u && dh != 0) atomicAdd(P.h00, (unsigned long long)(long long)dh);
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq)
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq) __stcg(w + (size_t)plane(yq, xq) * NR + R, T[yq][xq]);
}

// Sub-step i_sub of the sweep: every tile, from a work queue whose last fetch
// returns the counter to zero (as in the sweep kernel).
template <bool kGeneral>
__global__ void __launch_bounds__(256, 2) colour_kernel(const SweepParams P, uint32_t i_sub, uint32_t m) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  const uint32_t s = (uint32_t)(*P.t_dev) + P.s_add;
  const uint32_t cls = philox((kTagClass << 28) | i_sub, 0xffffffffu, s, P.sample, P.k0, P.k1).x & 3u;
  const uint32_t n = P.ntx * P.nty;
  uint32_t c = 0;
  if (lane == 0) c = atomicAdd(P.queue, 1u);
  c = __shfl_sync(kFull, c, 0);
  while (c < n) {
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(P.queue, 1u);
    colour_tile<kGeneral>(P, lane, s, i_sub, m, cls, c % P.ntx, c / P.ntx);
    c = __shfl_sync(kFull, next, 0);
  }
  if (lane == 0 && c == n + W - 1u) atomicExch(P.queue, 0u);
}

template <bool kGeneral>
cudaError_t launch_sub(const SweepParams& P, uint32_t i_sub, uint32_t m, cudaStream_t st) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static uint32_t cache[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  uint32_t ctas = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < kMaxDev && cache[dev]) {
      ctas = cache[dev];
    } else {
      int per_sm = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, colour_kernel<kGeneral>, 256, 0);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      ctas = (uint32_t)std::max(per_sm, 1) * (uint32_t)std::max(sms, 1);
      if (dev < kMaxDev) cache[dev] = ctas;
    }
  }
  const uint32_t tiles = P.ntx * P.nty;
  const uint32_t blocks = std::min<uint32_t>(ctas, (tiles + kWarps - 1u) / kWarps);
  colour_kernel<kGeneral><<<blocks, kWarps * 32u, 0, st>>>(P, i_sub, m);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_colour(const SweepParams& P, uint32_t m, cudaStream_t st) {
  if (m > 4u || P.nty * kTile != P.g.L) return cudaErrorInvalidValue;
  const bool general = !(P.Tp == 65536u && P.Tq == 0u);
  for (uint32_t i = 0; i < (4u << m); ++i) {
    const cudaError_t e = general ? launch_sub<true>(P, i, m, st) : launch_sub<false>(P, i, m, st);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  return cudaSuccess;
}

}  // namespace kpz
