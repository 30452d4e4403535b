// kpz_tile.cuh -- one warp sweeps a run of 128 x 128 tiles of one sweep.
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
// Mapping: one warp owns a tile (a run of tiles along x, processed in turn);
// lane l owns cell row l (tile rows 4l..4l+3). The tile lives in 16 registers
// per lane, one per site (x', y') of the 4 x 4 cell, bit c = cell c of the
// lane's cell row. A round evaluates the rule for the four sites of the active
// quadrant on all 32 cells at once with bitwise logic; neighbours in x come
// from a 1-bit shift (cells c-1, c+1), neighbours in y from the lanes above and
// below (warp shuffles). The right neighbour of the last cell column and the
// row below the last lane belong to the next tiles' dead borders, which no one
// changes during the sweep: they are read as halos. The next block column is
// copied into shared memory (cp.async, bypassing L1) while the current tile
// is processed.
#pragma once
#include "kpz_rounds.cuh"

namespace kpz {
namespace tile {

using rounds::TileCtx;
using rounds::tile_rounds;

// 16-byte asynchronous global -> shared copy that bypasses L1 (a persistent
// caller revisits lattice words other SMs changed since).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr uint32_t kSlab = 36;  // 4-row-aligned superset of the 32 (+1 halo) rows a plane needs

// Per-warp shared memory. Slab[slot][plane][row]: one block column, rows from
// the plane's 4-aligned base; M: per plane, the bits of the window's two block
// columns that lie outside the window.
struct alignas(16) WarpStage {
  uint32_t Slab[2][kPlanes][kSlab];
  uint32_t M[kPlanes][32];
};
static_assert((kSlab * 4) % 16 == 0, "slab rows must be whole 16-byte chunks");

// One warp sweeps tiles (ty, tx0 .. tx0 + P.run - 1) of sweep s of the lattice
// P describes (P is read in place: kernel parameter space or shared memory).
template <bool kGeneral>
__device__ __forceinline__ void run_tiles(const SweepParams& P, uint32_t s, uint32_t ty, uint32_t tx0,
                                          WarpStage& ws, uint32_t lane) {
  const uint32_t L = P.g.L, NR = P.g.NR, NB = P.g.NB;
  // Device layer: random origin of this sweep's tile grid.
  const uint4 o = philox(kTagOrigin << 28, 0u, s, P.sample, P.k0, P.k1);
  const uint32_t ox = o.x & (L - 1u), oy = o.y & (L - 1u);

  // Rows: tile row y' lives in storage cell row Rb + lane + cy(y'), plane row (by+y')%4.
  const uint32_t Y0 = (oy + ty * kTile) & (L - 1u);
  const uint32_t by = Y0 & 3u, Rb = Y0 >> 2;
  uint32_t rowR[4];  // storage cell row of lane 0's tile row y'; slab offset = rowR & 3
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq) rowR[yq] = (Rb + ((by + yq) >> 2)) & (NR - 1u);
  // Columns: tile column x' sits in storage column (bx+x')%4 starting at storage
  // cell column a + carry; its 32 cells are a 32-bit window at shift sh inside
  // two consecutive block columns.
  const uint32_t X0 = (ox + tx0 * kTile) & (L - 1u);
  const uint32_t bx = X0 & 3u, a = X0 >> 2;
  uint32_t shx[4], kx[4];
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t st = (a + ((bx + xq) >> 2)) & (L / 4u - 1u);
    shx[xq] = st & 31u;
    kx[xq] = st >> 5;
  }
  const size_t kstride = (size_t)kPlanes * NR;
  // storage plane of tile plane (x', y')
  auto splane = [&](uint32_t xq, uint32_t yq) -> uint32_t { return ((by + yq) & 3u) * 4u + ((bx + xq) & 3u); };
  // this lane's word of tile plane (x', y') in block column t of the run
  auto gword = [&](uint32_t xq, uint32_t yq, uint32_t t) -> uint32_t* {
    const uint32_t K = (kx[xq] + t) & (NB - 1u);
    return P.lat + (size_t)K * kstride + (size_t)splane(xq, yq) * NR +
           ((rowR[yq] + lane) & (NR - 1u));
  };
  // Queue the copy of block column t of the run into slab slot t & 1. Lane l
  // copies plane l % 16: lanes 0-15 its 16-byte chunks 0-4, lanes 16-31 its
  // chunks 5-8 (36 rows from the plane's 4-aligned first row).
  const uint32_t fp = lane & 15u, fx = fp & 3u, fy = fp >> 2;
  const uint32_t fch0 = lane < 16u ? 0u : 5u, fnch = lane < 16u ? 5u : 4u;
  const uint32_t fK0 = ((a + ((bx + fx) >> 2)) & (L / 4u - 1u)) >> 5;
  const size_t foff = (size_t)(((by + fy) & 3u) * 4u + ((bx + fx) & 3u)) * NR;
  const uint32_t frow0 = ((Rb + ((by + fy) >> 2)) & ~3u) + 4u * fch0;
  auto fetch = [&](uint32_t t) {
    const uint32_t* base = P.lat + (size_t)((fK0 + t) & (NB - 1u)) * kstride + foff;
    uint32_t* dst = &ws.Slab[t & 1u][fp][4u * fch0];
#pragma unroll
    for (uint32_t j = 0; j < 5u; ++j)
      if (j < fnch) cp_async16(dst + 4u * j, base + ((frow0 + 4u * j) & (NR - 1u)));
    cp_async_commit();
  };
  const bool last_lane = lane == 31u;
  const int par = (int)((X0 + Y0 + P.g.par) & 1u);

  uint32_t T[4][4], hy[4];
  // Prologue: block columns 0 and 1 form the first window.
  __syncwarp();
  fetch(0u);
  fetch(1u);
  cp_async_wait();
  __syncwarp();
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq)
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq) {
      const uint32_t p = yq * 4u + xq, low = (1u << shx[xq]) - 1u;
      const uint32_t C = ws.Slab[0][p][(rowR[yq] & 3u) + lane], N = ws.Slab[1][p][(rowR[yq] & 3u) + lane];
      T[yq][xq] = __funnelshift_r(C, N, shx[xq]);
      ws.M[p][lane] = (C & low) | (N & ~low);
    }
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq)  // row below the tile: y' = 0 planes, slab row + 32
    hy[xq] = __funnelshift_r(ws.Slab[0][xq][(rowR[0] & 3u) + 32u], ws.Slab[1][xq][(rowR[0] & 3u) + 32u], shx[xq]);
  __syncwarp();
  if (P.run > 1u) fetch(2u);

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

    // Right halo: column u = 128 (tile t+1's dead column), bit sh of M[x'=0].
    uint32_t hx[4];
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq) hx[yq] = (ws.M[yq * 4u][lane] >> shx[0]) & 1u;

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
    if (!last) {
      cp_async_wait();  // block column t+2 is in slot t & 1
      __syncwarp();
    }
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq)
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq) {
        const uint32_t p = yq * 4u + xq;
        const uint32_t sh = shx[xq];
        const uint32_t low = (1u << sh) - 1u;
        const uint32_t Tv = T[yq][xq], Mv = ws.M[p][lane];
        const uint32_t wl = (Mv & low) | (Tv << sh);                    // word t
        const uint32_t cn = (Mv & ~low) | __funnelshift_l(Tv, 0u, sh);  // word t+1
        uint32_t* pl = gword(xq, yq, t);
        if (t == 0u && sh != 0u) {
          // left word shared with the run to the left: xor in our bits only
          const uint32_t delta = (wl ^ __ldcg(pl)) & ~low;
          if (delta) atomicXor(pl, delta);
        } else {
          __stcg(pl, wl);
        }
        if (last) {
          if (sh != 0u) {  // right word shared with the run to the right
            uint32_t* pr = gword(xq, yq, t + 1u);
            const uint32_t delta = (cn ^ __ldcg(pr)) & low;
            if (delta) atomicXor(pr, delta);
          }
        } else {
          const uint32_t N = ws.Slab[t & 1u][p][(rowR[yq] & 3u) + lane];  // block column t+2
          T[yq][xq] = __funnelshift_r(cn, N, sh);
          ws.M[p][lane] = (cn & low) | (N & ~low);
        }
      }
    if (!last) {
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq)  // tile t+1's row below: block columns t+1, t+2
        hy[xq] = __funnelshift_r(ws.Slab[(t + 1u) & 1u][xq][(rowR[0] & 3u) + 32u],
                                 ws.Slab[t & 1u][xq][(rowR[0] & 3u) + 32u], shx[xq]);
      __syncwarp();
      if (t + 2u < P.run) fetch(t + 3u);   // for the end of tile t+1
    }
  }
  __syncwarp();
}

}  // namespace tile
}  // namespace kpz
