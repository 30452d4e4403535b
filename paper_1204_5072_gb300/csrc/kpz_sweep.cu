// kpz_sweep.cu -- one Monte Carlo sweep of the octahedron KPZ model on GB300.
//
// Decomposition (arXiv:1204.5072, Sec. 3 and 3.1):
//   device layer     -- 128 x 128 tiles whose grid origin (ox, oy) is redrawn
//                       every sweep; the low-x column and low-y row of a tile
//                       (its dead border) are never updated, so tiles do not
//                       interact and run concurrently;
//   work-group layer -- single-hit double tiling: each tile is split into
//                       4 x 4 cells, each cell into four 2 x 2 quadrants; in
//                       each of 16 rounds one random quadrant set is active
//                       and every cell makes one attempt at a random site of
//                       its active quadrant.
// Update rule: eq. (rule), Sec. 2.1 -- a site lower than its four neighbours
// rises by 2 with probability p, a site higher than all four drops by 2 with
// probability q. With the height bits of kpz_common.cuh a neighbour is higher
// iff its bit equals v = b(s) ^ parity(s); a minimum has all four neighbours
// equal to v, a maximum none; a move toggles b(s).
//
// Mapping: one warp owns a tile (a run of `run` tiles along x, processed in
// turn); lane l owns cell row l (tile rows 4l..4l+3). The tile lives in 16
// registers per lane, one per site (x', y') of the 4 x 4 cell, bit c = cell c
// of the lane's cell row. A round evaluates the rule for the four sites of the
// active quadrant on all 32 cells at once with bitwise logic; neighbours in x
// come from a 1-bit shift (cells c-1, c+1), neighbours in y from the lanes
// above and below (warp shuffles). The right neighbour of the last cell column
// and the row below the last lane belong to the next tiles' dead borders,
// which no one changes during the sweep: they are read once as halos.
// The next block column is copied into shared memory (cp.async) one tile ahead.
#include "kpz_rounds.cuh"

namespace kpz {
namespace {

using rounds::TileCtx;
using rounds::tile_rounds;

// Asynchronous 4-byte global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async4(uint32_t* smem, const uint32_t* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Per-warp staging in shared memory (each lane only touches its own column):
// M: per plane, the bits of the window's two block columns that lie outside
// the window; Pf: next block column, double-buffered; Hf: lane 31's halo row,
// a ring of three block columns.
struct WarpStage {
  uint32_t M[kPlanes][32];
  uint32_t Pf[2][kPlanes][32];
  uint32_t Hf[3][4];
};
constexpr uint32_t kWarpsPerCta = 8;

template <bool kGeneral>
__global__ void __launch_bounds__(256, kGeneral ? 2 : 3) sweep_kernel(const SweepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpStage& ws = reinterpret_cast<WarpStage*>(smem_raw)[threadIdx.x >> 5];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= P.runs_x * P.nty) return;
  const uint32_t ty = gw / P.runs_x;
  const uint32_t tx0 = (gw - ty * P.runs_x) * P.run;
  const uint32_t L = P.g.L, NR = P.g.NR, NB = P.g.NB;
  const uint32_t s = (uint32_t)(*P.t_dev) + P.s_add;

  // Device layer: random origin of this sweep's tile grid.
  const uint4 o = philox(kTagOrigin << 28, 0u, s, P.sample, P.k0, P.k1);
  const uint32_t ox = o.x & (L - 1u), oy = o.y & (L - 1u);

  // Rows: tile row y' of this lane lives in storage cell row rowR, plane row (by+y')%4.
  const uint32_t Y0 = (oy + ty * kTile) & (L - 1u);
  const uint32_t by = Y0 & 3u, Rb = Y0 >> 2;
  uint32_t offY[4];
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq)
    offY[yq] = ((by + yq) & 3u) * 4u * NR + ((Rb + lane + ((by + yq) >> 2)) & (NR - 1u));
  const uint32_t offH = by * 4u * NR + ((Rb + 32u) & (NR - 1u));  // row below the tile (y' = 0)
  // Columns: tile column x' sits in storage column (bx+x')%4 starting at storage
  // cell column a + carry; its 32 cells are a 32-bit window at shift sh inside
  // two consecutive block columns.
  const uint32_t X0 = (ox + tx0 * kTile) & (L - 1u);
  const uint32_t bx = X0 & 3u, a = X0 >> 2;
  uint32_t offX[4], shx[4], kx[4];
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t st = (a + ((bx + xq) >> 2)) & (L / 4u - 1u);
    offX[xq] = ((bx + xq) & 3u) * NR;
    shx[xq] = st & 31u;
    kx[xq] = st >> 5;
  }
  const size_t kstride = (size_t)kPlanes * NR;
  auto col = [&](uint32_t xq, uint32_t t) -> uint32_t* {
    return P.lat + (size_t)((kx[xq] + t) & (NB - 1u)) * kstride + offX[xq];
  };
  const bool last_lane = lane == 31u;
  const int par = (int)((X0 + Y0 + P.g.par) & 1u);
  // Queue the copies of block column t into the staging slots.
  auto prefetch = [&](uint32_t t) {
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq) {
      const uint32_t* c = col(xq, t);
#pragma unroll
      for (uint32_t yq = 0; yq < 4; ++yq) cp_async4(&ws.Pf[t & 1u][yq * 4 + xq][lane], c + offY[yq]);
      if (last_lane) cp_async4(&ws.Hf[t % 3u][xq], c + offH);
    }
    cp_async_commit();
  };

  uint32_t T[4][4];
  // Prologue: window of the first tile (block columns 0 and 1).
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t* c0 = col(xq, 0);
    const uint32_t* c1 = col(xq, 1);
    const uint32_t low = (1u << shx[xq]) - 1u;
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq) {
      const uint32_t C = __ldcg(c0 + offY[yq]);
      const uint32_t N = __ldcg(c1 + offY[yq]);
      T[yq][xq] = __funnelshift_r(C, N, shx[xq]);
      ws.M[yq * 4 + xq][lane] = (C & low) | (N & ~low);
    }
    if (last_lane) {
      ws.Hf[0][xq] = __ldcg(c0 + offH);
      ws.Hf[1][xq] = __ldcg(c1 + offH);
    }
  }
  if (P.run > 1u) prefetch(2u);

  TileCtx tc;
  tc.s = s;
  tc.first_row_ok = lane == 0u ? 0u : ~0u;
  tc.last_lane = last_lane;
  const uint32_t vo = (0u - Y0) & (L - 1u);

#pragma unroll 1
  for (uint32_t t = 0; t < P.run; ++t) {
    tc.tid = ty * P.ntx + tx0 + t;
    tc.setw = philox(kTagSet << 28, tc.tid, s, P.sample, P.k0, P.k1).x;
    const uint32_t uo = (0u - ((X0 + t * kTile) & (L - 1u))) & (L - 1u);
    tc.track = (uo < kTile) && (vo < kTile);
    tc.xo = uo & 3u; tc.co = uo >> 2; tc.yo = vo & 3u; tc.cyo = vo >> 2;

    // Halos: column u = 128 (tile t+1's dead column) and, for lane 31, row v = 128.
    uint32_t hx[4], hy[4];
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq) hx[yq] = (ws.M[yq * 4][lane] >> shx[0]) & 1u;
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq)
      hy[xq] = last_lane ? __funnelshift_r(ws.Hf[t % 3u][xq], ws.Hf[(t + 1u) % 3u][xq], shx[xq]) : 0u;

    int dh = 0;
    // The one tile per sweep that holds site (0,0) also counts its moves.
    if (tc.track) {
      if (par) tile_rounds<kGeneral, 1, true>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, true>(T, hx, hy, P, tc, lane, dh);
    } else {
      if (par) tile_rounds<kGeneral, 1, false>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, false>(T, hx, hy, P, tc, lane, dh);
    }
    if (tc.track && lane == tc.cyo && dh != 0)
      atomicAdd(P.h00, (unsigned long long)(long long)dh);

    // Write back block column t and slide the window to tile t+1.
    const bool last = (t + 1u == P.run);
    cp_async_wait();
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq) {
      const uint32_t sh = shx[xq];
      const uint32_t low = (1u << sh) - 1u;
      uint32_t* cl = col(xq, t);
      uint32_t* cr = col(xq, t + 1u);
#pragma unroll
      for (uint32_t yq = 0; yq < 4; ++yq) {
        const uint32_t Tv = T[yq][xq], Mv = ws.M[yq * 4 + xq][lane];
        const uint32_t wl = (Mv & low) | (Tv << sh);                    // word t
        const uint32_t cn = (Mv & ~low) | __funnelshift_l(Tv, 0u, sh);  // word t+1
        uint32_t* pl = cl + offY[yq];
        if (t == 0u && sh != 0u) {
          // left word shared with the run to the left: xor in our bits only
          const uint32_t delta = (wl ^ __ldcg(pl)) & ~low;
          if (delta) atomicXor(pl, delta);
        } else {
          __stcg(pl, wl);
        }
        if (last) {
          if (sh != 0u) {  // right word shared with the run to the right
            uint32_t* pr = cr + offY[yq];
            const uint32_t delta = (cn ^ __ldcg(pr)) & low;
            if (delta) atomicXor(pr, delta);
          }
        } else {
          const uint32_t N = ws.Pf[t & 1u][yq * 4 + xq][lane];  // block column t+2
          T[yq][xq] = __funnelshift_r(cn, N, sh);
          ws.M[yq * 4 + xq][lane] = (cn & low) | (N & ~low);
        }
      }
    }
    if (t + 2u < P.run) prefetch(t + 3u);   // for the end of tile t+1
  }
}

__global__ void advance_kernel(uint64_t* t_dev, uint32_t n) { *t_dev += n; }

}  // namespace

cudaError_t launch_sweep(const SweepParams& P, uint32_t warps_per_cta, cudaStream_t st) {
  const uint64_t warps = (uint64_t)P.runs_x * P.nty;
  const uint32_t wpc = warps_per_cta ? warps_per_cta : 8u;
  const uint64_t blocks = (warps + wpc - 1) / wpc;
  const size_t smem = wpc * sizeof(WarpStage);
  static bool attr_set = false;   // opt in to more than 48 KB of dynamic shared memory once
  if (!attr_set) {
    const int bytes = (int)(kWarpsPerCta * sizeof(WarpStage));
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const bool general = !(P.Tp == 65536u && P.Tq == 0u);
  if (general)
    sweep_kernel<true><<<(unsigned)blocks, wpc * 32u, smem, st>>>(P);
  else
    sweep_kernel<false><<<(unsigned)blocks, wpc * 32u, smem, st>>>(P);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_advance(uint64_t* t_dev, uint32_t n, cudaStream_t st) {
  advance_kernel<<<1, 1, 0, st>>>(t_dev, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kpz
