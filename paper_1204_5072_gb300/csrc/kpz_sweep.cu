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
// The next block column is prefetched into registers one tile ahead.
#include "kpz_internal.h"

namespace kpz {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

struct TileCtx {
  uint32_t tid;           // tile id ty*ntx + tx (Philox counter word 1)
  uint32_t s;             // sweep index (Philox counter word 2)
  uint32_t setw;          // 16 x 2 bits: quadrant set of each round
  uint32_t first_row_ok;  // ~0 unless lane 0 (tile row v = 0 is dead)
  bool last_lane;         // lane 31: the row below comes from the halo
  bool track;             // this tile contains site (0,0)
  uint32_t xo, yo, co, cyo;  // position of site (0,0) in the tile
};

// Bit-serial comparison U < T for the 32 cells of a lane (U uniform 16-bit,
// level n = bit 15-n of U taken from bit c of word n&3 of Philox call n>>2).
// Only cells in needp (selected site is a minimum) and needq (a maximum) need
// a decision; a cell is decided at the first level where U and T differ, so
// the warp stops drawing levels once no cell of any lane is still tied. The
// outcome equals the full 16-level comparison.
__device__ __forceinline__ void acceptance(const SweepParams& P, const TileCtx& tc, uint32_t lane,
                                           uint32_t r, uint32_t needp, uint32_t needq,
                                           uint32_t& AP, uint32_t& AQ) {
  uint32_t ltp = 0u, ltq = 0u;
  uint32_t undp = (P.Tp == 0u || (P.Tp >> 16)) ? 0u : needp;
  uint32_t undq = (P.Tq == 0u || (P.Tq >> 16)) ? 0u : needq;
#pragma unroll 1
  for (uint32_t m = 0; m < 4; ++m) {
    if (4u * m >= P.nlev || !__any_sync(0xffffffffu, (undp | undq) != 0u)) break;
    const uint4 A = philox((kTagAcc << 28) | (lane << 6) | (r << 2) | m, tc.tid, tc.s, P.sample,
                           P.k0, P.k1);
    const uint32_t w[4] = {A.x, A.y, A.z, A.w};
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t n = 4u * m + j;
      const uint32_t bp = 0u - ((P.Tp >> (15u - n)) & 1u);
      const uint32_t bq = 0u - ((P.Tq >> (15u - n)) & 1u);
      ltp |= undp & ~w[j] & bp;
      undp &= ~(w[j] ^ bp);
      ltq |= undq & ~w[j] & bq;
      undq &= ~(w[j] ^ bq);
    }
  }
  AP = (P.Tp >> 16) ? ~0u : ltp;
  AQ = (P.Tq >> 16) ? ~0u : ltq;
}

// One single-hit round with active quadrant (QX, QY); kPar = parity of the
// tile's site (0,0). T[y'][x'], hx[y'] (bit 0: right halo), hy[x'] (lane 31:
// the row below the tile).
template <int QX, int QY, bool kGeneral, int kPar, bool kTrack>
__device__ __forceinline__ void quad_round(uint32_t (&T)[4][4], uint32_t Xi, uint32_t Yi,
                                           const uint32_t (&hx)[4], const uint32_t (&hy)[4],
                                           const SweepParams& P, const TileCtx& tc,
                                           uint32_t lane, uint32_t r, int& dh) {
  constexpr int x0 = 2 * QX, y0 = 2 * QY;
  uint32_t sel[2][2];  // [dy][dx]: cells whose random site is (x0+dx, y0+dy)
  sel[0][0] = ~Xi & ~Yi;
  sel[0][1] = Xi & ~Yi;
  sel[1][0] = ~Xi & Yi;
  sel[1][1] = Xi & Yi;
  if (QX == 0) { sel[0][0] &= ~1u; sel[1][0] &= ~1u; }       // tile column u = 0
  if (QY == 0) { sel[0][0] &= tc.first_row_ok; sel[0][1] &= tc.first_row_ok; }  // row v = 0

  uint32_t xn[2], yn[2];  // neighbours outside the cell (x) and outside the lane (y)
#pragma unroll
  for (int d = 0; d < 2; ++d)
    xn[d] = (QX == 0) ? (T[y0 + d][3] << 1)                            // cell c-1, column 3
                      : __funnelshift_r(T[y0 + d][0], hx[y0 + d], 1);  // cell c+1, column 0
  if (QY == 0) {
    yn[0] = __shfl_up_sync(kFull, T[3][x0], 1);
    yn[1] = __shfl_up_sync(kFull, T[3][x0 + 1], 1);
  } else {
    const uint32_t d0 = __shfl_down_sync(kFull, T[0][x0], 1);
    const uint32_t d1 = __shfl_down_sync(kFull, T[0][x0 + 1], 1);
    yn[0] = tc.last_lane ? hy[x0] : d0;
    yn[1] = tc.last_lane ? hy[x0 + 1] : d1;
  }

  uint32_t fmin[2][2], fmax[2][2];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int xp = x0 + dx, yp = y0 + dy;
      const uint32_t s = T[yp][xp];
      const uint32_t nL = (xp > 0) ? T[yp][xp > 0 ? xp - 1 : 0] : xn[dy];
      const uint32_t nR = (xp < 3) ? T[yp][xp < 3 ? xp + 1 : 3] : xn[dy];
      const uint32_t nU = (yp > 0) ? T[yp > 0 ? yp - 1 : 0][xp] : yn[dx];
      const uint32_t nD = (yp < 3) ? T[yp < 3 ? yp + 1 : 3][xp] : yn[dx];
      const uint32_t v = ((kPar + xp + yp) & 1) ? ~s : s;   // bit of a higher neighbour
      const uint32_t hL = ~(nL ^ v), hR = ~(nR ^ v), hU = ~(nU ^ v), hD = ~(nD ^ v);
      fmin[dy][dx] = sel[dy][dx] & hL & hR & hU & hD;                       // local minimum
      fmax[dy][dx] = kGeneral ? (sel[dy][dx] & ~hL & ~hR & ~hU & ~hD) : 0u;  // local maximum
    }
  if (kGeneral) {
    uint32_t AP, AQ;
    acceptance(P, tc, lane, r, fmin[0][0] | fmin[0][1] | fmin[1][0] | fmin[1][1],
               fmax[0][0] | fmax[0][1] | fmax[1][0] | fmax[1][1], AP, AQ);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) { fmin[dy][dx] &= AP; fmax[dy][dx] &= AQ; }
  }
  if (kTrack && lane == tc.cyo) {
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
        if ((uint32_t)(x0 + dx) == tc.xo && (uint32_t)(y0 + dy) == tc.yo)
          dh += 2 * (int)((fmin[dy][dx] >> tc.co) & 1u) - 2 * (int)((fmax[dy][dx] >> tc.co) & 1u);
  }
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) T[y0 + dy][x0 + dx] ^= fmin[dy][dx] | fmax[dy][dx];
}

template <bool kGeneral, int kPar, bool kTrack>
__device__ __forceinline__ void one_round(uint32_t (&T)[4][4], uint32_t Xi, uint32_t Yi,
                                          const uint32_t (&hx)[4], const uint32_t (&hy)[4],
                                          const SweepParams& P, const TileCtx& tc, uint32_t lane,
                                          uint32_t r, int& dh) {
  switch ((tc.setw >> (2u * r)) & 3u) {
    case 0: quad_round<0, 0, kGeneral, kPar, kTrack>(T, Xi, Yi, hx, hy, P, tc, lane, r, dh); break;
    case 1: quad_round<1, 0, kGeneral, kPar, kTrack>(T, Xi, Yi, hx, hy, P, tc, lane, r, dh); break;
    case 2: quad_round<0, 1, kGeneral, kPar, kTrack>(T, Xi, Yi, hx, hy, P, tc, lane, r, dh); break;
    default: quad_round<1, 1, kGeneral, kPar, kTrack>(T, Xi, Yi, hx, hy, P, tc, lane, r, dh); break;
  }
}

// The 16 single-hit rounds of one tile, two rounds per Philox block of positions.
template <bool kGeneral, int kPar, bool kTrack>
__device__ __forceinline__ void tile_rounds(uint32_t (&T)[4][4], const uint32_t (&hx)[4],
                                         const uint32_t (&hy)[4], const SweepParams& P,
                                         const TileCtx& tc, uint32_t lane, int& dh) {
#pragma unroll 1
  for (uint32_t rp = 0; rp < kRounds / 2; ++rp) {
    const uint4 pos = philox((kTagPos << 28) | (lane << 3) | rp, tc.tid, tc.s, P.sample, P.k0, P.k1);
    one_round<kGeneral, kPar, kTrack>(T, pos.x, pos.y, hx, hy, P, tc, lane, 2u * rp, dh);
    one_round<kGeneral, kPar, kTrack>(T, pos.z, pos.w, hx, hy, P, tc, lane, 2u * rp + 1u, dh);
  }
}

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
