// kpz_tileset.cu -- one sweep of the tile-set variant of the device layer.
//
// The paper decomposes the KPZ lattice with dead-border tiles (Sec. 3) and
// describes, for its KMC model, a double tiling at the device layer instead:
// the tiles form four sets, the sets are swept one after the other in an
// order drawn per sweep, and the tiles of one set are never neighbours, so
// they need no dead border (Sec. 3.2). This file implements that variant for
// the KPZ model: the same random origin and 128 x 128 tiles as the
// dead-border sweep, set (tx & 1) + 2 (ty & 1), four launches per sweep (one
// per set, in the drawn order), every site of a tile live, and the same
// work-group layer (16 single-hit rounds, kpz_rounds.cuh) and random streams.
//
// A warp takes one tile of the current set at a time from a work queue. It
// loads the tile's window (two block columns per plane), the column left of
// the tile, the row above (lane 0) and the row below (lane 31); the tiles
// around it are idle during this launch, so their bits are constant and the
// window's words are written back whole.
#include <algorithm>
#include <mutex>

#include "kpz_internal.h"
#include "kpz_rounds.cuh"

namespace kpz {
namespace {

using rounds::kFull;
using rounds::TileCtx;
using rounds::tile_rounds;

constexpr uint32_t kWarps = 8;

// Set swept in phase `phase` of sweep s: a Fisher-Yates shuffle of (0,1,2,3)
// driven by philox(5 << 28, 0, s, sample).
__device__ __forceinline__ uint32_t phase_set(const SweepParams& P, uint32_t s, uint32_t phase) {
  const uint4 w = philox(kTagPhase << 28, 0u, s, P.sample, P.k0, P.k1);
  uint32_t perm[4] = {0u, 1u, 2u, 3u};
  const uint32_t r[3] = {w.x, w.y, w.z};
#pragma unroll
  for (uint32_t i = 3; i >= 1; --i) {
    const uint32_t j = r[3 - i] % (i + 1u), t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  return perm[phase & 3u];
}

template <bool kGeneral>
__device__ __forceinline__ void tileset_tile(const SweepParams& P, uint32_t (&Mw)[kPlanes][32],
                                             uint32_t lane, uint32_t s, uint32_t ox, uint32_t oy,
                                             uint32_t tx, uint32_t ty) {
  const uint32_t L = P.g.L, NR = P.g.NR, NB = P.g.NB;
  const uint32_t Y0 = (oy + ty * kTile) & (L - 1u), X0 = (ox + tx * kTile) & (L - 1u);
  const uint32_t by = Y0 & 3u, Rb = Y0 >> 2, bx = X0 & 3u, a = X0 >> 2;
  uint32_t offY[4];
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq)
    offY[yq] = ((by + yq) & 3u) * 4u * NR + ((Rb + lane + ((by + yq) >> 2)) & (NR - 1u));
  const uint32_t offH = by * 4u * NR + ((Rb + 32u) & (NR - 1u));                        // row below
  const uint32_t offU = ((by + 3u) & 3u) * 4u * NR + ((Rb - 1u + ((by + 3u) >> 2)) & (NR - 1u));  // row above
  uint32_t shx[4];
  const uint32_t* cl[4];
  uint32_t* wl[4];
  uint32_t* wr[4];
  const size_t kstride = (size_t)kPlanes * NR;
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t st = (a + ((bx + xq) >> 2)) & (L / 4u - 1u);
    const uint32_t kx = st >> 5, offX = ((bx + xq) & 3u) * NR;
    shx[xq] = st & 31u;
    wl[xq] = P.lat + (size_t)kx * kstride + offX;
    wr[xq] = P.lat + (size_t)((kx + 1u) & (NB - 1u)) * kstride + offX;
    cl[xq] = P.lat + (size_t)((kx + NB - 1u) & (NB - 1u)) * kstride + offX;   // block column before
  }
  const bool first_lane = lane == 0u, last_lane = lane == 31u;
  TileCtx tc;
  uint32_t T[4][4], hx[4], hy[4];
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t sh = shx[xq], low = (1u << sh) - 1u;
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq) {
      const uint32_t C = __ldcg(wl[xq] + offY[yq]), N = __ldcg(wr[xq] + offY[yq]);
      T[yq][xq] = __funnelshift_r(C, N, sh);
      Mw[yq * 4 + xq][lane] = (C & low) | (N & ~low);
      if (xq == 3) {   // the site left of the tile: cell before the window's first cell, column 3
        const uint32_t B = sh ? C : __ldcg(cl[xq] + offY[yq]);
        tc.hxl[yq] = (B >> ((sh + 31u) & 31u)) & 1u;
      }
      if (xq == 0) hx[yq] = (N >> sh) & 1u;   // the site right of the tile (column 0 of cell 32)
    }
    hy[xq] = last_lane ? __funnelshift_r(__ldcg(wl[xq] + offH), __ldcg(wr[xq] + offH), sh) : 0u;
    tc.hyu[xq] = first_lane ? __funnelshift_r(__ldcg(wl[xq] + offU), __ldcg(wr[xq] + offU), sh) : 0u;
  }
  const int par = (int)((X0 + Y0 + P.g.par) & 1u);
  tc.tid = ty * P.ntx + tx;
  tc.s = s;
  tc.setw = philox(kTagSet << 28, tc.tid, s, P.sample, P.k0, P.k1).x;
  tc.first_row_ok = first_lane ? 0u : ~0u;
  tc.last_lane = last_lane;
  tc.rk = nullptr;
  tc.pm = par ? ~0u : 0u;
  const uint32_t uo = (0u - X0) & (L - 1u), vo = (0u - Y0) & (L - 1u);
  tc.track = (uo < kTile) && (vo < kTile);
  tc.xo = uo & 3u; tc.co = uo >> 2; tc.yo = vo & 3u; tc.cyo = vo >> 2;
  uint32_t T1[1][4][4], hx1[1][4];
#pragma unroll
  for (uint32_t y = 0; y < 4; ++y)
#pragma unroll
    for (uint32_t x = 0; x < 4; ++x) T1[0][y][x] = T[y][x];
#pragma unroll
  for (uint32_t y = 0; y < 4; ++y) hx1[0][y] = hx[y];
  int dh = 0;
  if (tc.track) tile_rounds<kGeneral, 2, true, 1, false, true>(T1, hx1, hy, P, tc, lane, dh);
  else          tile_rounds<kGeneral, 2, false, 1, false, true>(T1, hx1, hy, P, tc, lane, dh);
  if (tc.track && lane == tc.cyo && dh != 0) atomicAdd(P.h00, (unsigned long long)(long long)dh);
  // Write the window back: the neighbouring tiles are idle, so whole words.
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t sh = shx[xq], low = (1u << sh) - 1u;
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq) {
      const uint32_t Tv = T1[0][yq][xq], Mv = Mw[yq * 4 + xq][lane];
      __stcg(wl[xq] + offY[yq], (Mv & low) | (Tv << sh));
      if (sh) __stcg(wr[xq] + offY[yq], (Mv & ~low) | __funnelshift_l(Tv, 0u, sh));
    }
  }
}

// One phase of one sweep: the tiles of the set drawn for `phase`, from a work
// queue whose last fetch returns the counter to zero (as in the sweep kernel).
template <bool kGeneral>
__global__ void __launch_bounds__(256, 2) tileset_kernel(const SweepParams P, uint32_t phase) {
  __shared__ uint32_t M[kWarps][kPlanes][32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  const uint32_t L = P.g.L;
  const uint32_t s = (uint32_t)(*P.t_dev) + P.s_add;
  const uint4 o = philox(kTagOrigin << 28, 0u, s, P.sample, P.k0, P.k1);
  const uint32_t ox = o.x & (L - 1u), oy = o.y & (L - 1u);
  const uint32_t set = phase_set(P, s, phase);
  const uint32_t hx_tiles = P.ntx / 2u, n = hx_tiles * (P.nty / 2u);
  uint32_t c = 0;
  if (lane == 0) c = atomicAdd(P.queue, 1u);
  c = __shfl_sync(kFull, c, 0);
  while (c < n) {
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(P.queue, 1u);
    const uint32_t iy = c / hx_tiles, ix = c - iy * hx_tiles;
    tileset_tile<kGeneral>(P, M[warp], lane, s, ox, oy, 2u * ix + (set & 1u), 2u * iy + (set >> 1));
    c = __shfl_sync(kFull, next, 0);
  }
  if (lane == 0 && c == n + W - 1u) atomicExch(P.queue, 0u);
}

template <bool kGeneral>
cudaError_t launch_phase(const SweepParams& P, uint32_t phase, cudaStream_t st) {
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
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tileset_kernel<kGeneral>, 256, 0);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      ctas = (uint32_t)std::max(per_sm, 1) * (uint32_t)std::max(sms, 1);
      if (dev < kMaxDev) cache[dev] = ctas;
    }
  }
  const uint32_t tiles = (P.ntx / 2u) * (P.nty / 2u);
  const uint32_t blocks = std::min<uint32_t>(ctas, (tiles + kWarps - 1u) / kWarps);
  tileset_kernel<kGeneral><<<blocks, kWarps * 32u, 0, st>>>(P, phase);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_tilesets(const SweepParams& P, cudaStream_t st) {
  if (P.nty * kTile != P.g.L || P.ntx < 2u || P.nty < 2u) return cudaErrorInvalidValue;
  const bool general = !(P.Tp == 65536u && P.Tq == 0u);
  for (uint32_t phase = 0; phase < 4; ++phase) {
    const cudaError_t e = general ? launch_phase<true>(P, phase, st) : launch_phase<false>(P, phase, st);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  return cudaSuccess;
}

}  // namespace kpz
