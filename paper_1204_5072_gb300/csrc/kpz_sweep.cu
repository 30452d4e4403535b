// kpz_sweep.cu -- one Monte Carlo sweep of the octahedron KPZ model on GB300.
//
// Decomposition (arXiv:1204.5072, Sec. 3 and 3.1):
//   device layer     -- 128 x 128 tiles whose grid origin (ox, oy) is redrawn
//                       every sweep; the low-x column and low-y row of a tile
//                       (its dead border) are never updated, so tiles touch
//                       disjoint slope bits and run concurrently;
//   work-group layer -- single-hit double tiling: each tile is split into
//                       4 x 4 cells, each cell into four 2 x 2 quadrants; in
//                       each of 16 rounds one random quadrant set is active
//                       and every cell makes one attempt at a random site of
//                       its active quadrant.
// Update rule: eq. (rule), Sec. 2.1.
//
// Mapping: one warp owns a tile (a run of `run` tiles along x, processed in
// turn); lane l owns cell row l (tile rows 4l..4l+3). The tile is held in 32
// registers per lane, one per (row y', column x', slope sigma) of the 4 x 4
// cell, bit c = cell c of the lane's cell row. A round evaluates the rule for
// the four sites of the active quadrant on all 32 cells at once with bitwise
// logic; neighbours in x come from a 1-bit shift (cell c-1), neighbours in y
// from the lane above (warp shuffle). Nothing is staged in shared memory.
#include "kpz_internal.h"

namespace kpz {
namespace {

struct TileCtx {
  uint32_t tid;           // tile id ty*ntx + tx (Philox counter word 1)
  uint32_t s;             // sweep index (Philox counter word 2)
  uint32_t setw;          // 16 x 2 bits: quadrant set of each round
  uint32_t first_row_ok;  // ~0 unless lane 0 (tile row v = 0 is dead)
  uint32_t last_row_ok;   // ~0 unless lane 31 (no lane below inside the tile)
  bool track;             // this tile contains site (0,0)
  uint32_t xo, yo, co, cyo;  // position of site (0,0) in the tile
};

// Bit-serial comparison U < T for the 32 cells of a lane (U uniform 16-bit,
// level n = bit 15-n of U taken from bit c of word n&3 of Philox call n>>2).
__device__ __forceinline__ void acceptance(const SweepParams& P, const TileCtx& tc, uint32_t lane,
                                           uint32_t r, uint32_t& AP, uint32_t& AQ) {
  uint32_t ltp = 0u, ltq = 0u, undp = ~0u, undq = ~0u;
#pragma unroll
  for (uint32_t m = 0; m < 4; ++m) {
    if (4u * m >= P.nlev) break;
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

// One single-hit round with active quadrant (QX, QY). T[y'][x'][sigma].
template <int QX, int QY, bool kGeneral>
__device__ __forceinline__ void quad_round(uint32_t (&T)[4][4][2], uint32_t Xi, uint32_t Yi,
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

  uint32_t left[2] = {0u, 0u}, up[2] = {0u, 0u};
  if (QX == 0) {  // x-slope leaving cell c-1 at its column 3
    left[0] = T[y0][3][0] << 1;
    left[1] = T[y0 + 1][3][0] << 1;
  }
  if (QY == 0) {  // y-slope leaving the lane above at its row 3
    up[0] = __shfl_up_sync(0xffffffffu, T[3][x0][1], 1);
    up[1] = __shfl_up_sync(0xffffffffu, T[3][x0 + 1][1], 1);
  }

  uint32_t fmin[2][2], fmax[2][2];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int xp = x0 + dx, yp = y0 + dy;
      const uint32_t a = (xp > 0) ? T[yp][xp > 0 ? xp - 1 : 0][0] : left[dy];
      const uint32_t b = T[yp][xp][0];
      const uint32_t c = (yp > 0) ? T[yp > 0 ? yp - 1 : 0][xp][1] : up[dx];
      const uint32_t d = T[yp][xp][1];
      fmin[dy][dx] = sel[dy][dx] & ~a & b & ~c & d;              // local minimum
      fmax[dy][dx] = kGeneral ? (sel[dy][dx] & a & ~b & c & ~d)  // local maximum
                              : 0u;
    }
  if (kGeneral) {
    uint32_t AP, AQ;
    acceptance(P, tc, lane, r, AP, AQ);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) { fmin[dy][dx] &= AP; fmax[dy][dx] &= AQ; }
  }
  if (tc.track && lane == tc.cyo) {
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
        if ((uint32_t)(x0 + dx) == tc.xo && (uint32_t)(y0 + dy) == tc.yo)
          dh += 2 * (int)((fmin[dy][dx] >> tc.co) & 1u) - 2 * (int)((fmax[dy][dx] >> tc.co) & 1u);
  }

  uint32_t down[2] = {0u, 0u};
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int xp = x0 + dx, yp = y0 + dy;
      const uint32_t f = fmin[dy][dx] | fmax[dy][dx];
      T[yp][xp][0] ^= f;
      T[yp][xp][1] ^= f;
      if (xp > 0) T[yp][xp > 0 ? xp - 1 : 0][0] ^= f;
      else        T[yp][3][0] ^= f >> 1;           // bit 0 is dead: nothing leaves the tile
      if (yp > 0) T[yp > 0 ? yp - 1 : 0][xp][1] ^= f;
      else        down[dx] = f;
    }
  if (QY == 0) {
    T[3][x0][1] ^= __shfl_down_sync(0xffffffffu, down[0], 1) & tc.last_row_ok;
    T[3][x0 + 1][1] ^= __shfl_down_sync(0xffffffffu, down[1], 1) & tc.last_row_ok;
  }
}

template <bool kGeneral>
__device__ __forceinline__ void one_round(uint32_t (&T)[4][4][2], uint32_t Xi, uint32_t Yi,
                                          const SweepParams& P, const TileCtx& tc, uint32_t lane,
                                          uint32_t r, int& dh) {
  switch ((tc.setw >> (2u * r)) & 3u) {
    case 0: quad_round<0, 0, kGeneral>(T, Xi, Yi, P, tc, lane, r, dh); break;
    case 1: quad_round<1, 0, kGeneral>(T, Xi, Yi, P, tc, lane, r, dh); break;
    case 2: quad_round<0, 1, kGeneral>(T, Xi, Yi, P, tc, lane, r, dh); break;
    default: quad_round<1, 1, kGeneral>(T, Xi, Yi, P, tc, lane, r, dh); break;
  }
}

template <bool kGeneral>
__global__ void __launch_bounds__(256, 2) sweep_kernel(const SweepParams P) {
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

  // Rows of this lane: tile row y' lives in storage cell row rowR, plane row rowY.
  const uint32_t Y0 = (oy + ty * kTile) & (L - 1u);
  const uint32_t by = Y0 & 3u, Rb = Y0 >> 2;
  uint32_t offY[4];  // word offset of (plane row, cell row) without column terms
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq) {
    const uint32_t rowR = (Rb + lane + ((by + yq) >> 2)) & (NR - 1u);
    const uint32_t rowY = (by + yq) & 3u;
    offY[yq] = rowY * 8u * NR + rowR;
  }
  // Columns: tile column x' sits in storage column (bx+x')%4, starting at
  // storage cell column a + carry; its 32 cells are a 32-bit window shifted
  // by sh inside two consecutive block columns.
  const uint32_t X0 = (ox + tx0 * kTile) & (L - 1u);
  const uint32_t bx = X0 & 3u, a = X0 >> 2;
  uint32_t offX[4], shx[4], kx[4];
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t st = (a + ((bx + xq) >> 2)) & (L / 4u - 1u);
    offX[xq] = ((bx + xq) & 3u) * 2u * NR;
    shx[xq] = st & 31u;
    kx[xq] = st >> 5;
  }
  const size_t kstride = (size_t)32u * NR;  // words between block columns
  auto addr = [&](uint32_t xq, uint32_t yq, uint32_t sg, uint32_t t) -> uint32_t* {
    const uint32_t K = (kx[xq] + t) & (NB - 1u);
    return P.lat + (size_t)K * kstride + offX[xq] + offY[yq] + sg * NR;
  };

  uint32_t T[4][4][2], M[4][4][2];
  // Prologue: window of the first tile. M keeps, per plane, the bits of the
  // two block columns that are not in the window (low part of the left word,
  // high part of the right word).
#pragma unroll
  for (uint32_t yq = 0; yq < 4; ++yq)
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq)
#pragma unroll
      for (uint32_t sg = 0; sg < 2; ++sg) {
        const uint32_t C = __ldcg(addr(xq, yq, sg, 0));
        const uint32_t N = __ldcg(addr(xq, yq, sg, 1));
        const uint32_t low = (1u << shx[xq]) - 1u;
        T[yq][xq][sg] = __funnelshift_r(C, N, shx[xq]);
        M[yq][xq][sg] = (C & low) | (N & ~low);
      }

  TileCtx tc;
  tc.s = s;
  tc.first_row_ok = lane == 0u ? 0u : ~0u;
  tc.last_row_ok = lane == 31u ? 0u : ~0u;
  const uint32_t vo = (0u - Y0) & (L - 1u);

  for (uint32_t t = 0; t < P.run; ++t) {
    const uint32_t tx = tx0 + t;
    tc.tid = ty * P.ntx + tx;
    tc.setw = philox(kTagSet << 28, tc.tid, s, P.sample, P.k0, P.k1).x;
    const uint32_t uo = (0u - ((X0 + t * kTile) & (L - 1u))) & (L - 1u);
    tc.track = (uo < kTile) && (vo < kTile);
    tc.xo = uo & 3u; tc.co = uo >> 2; tc.yo = vo & 3u; tc.cyo = vo >> 2;
    int dh = 0;

    // Work-group layer: 16 single-hit rounds, two per Philox block of positions.
#pragma unroll 1
    for (uint32_t rp = 0; rp < kRounds / 2; ++rp) {
      const uint4 pos = philox((kTagPos << 28) | (lane << 3) | rp, tc.tid, s, P.sample, P.k0, P.k1);
      one_round<kGeneral>(T, pos.x, pos.y, P, tc, lane, 2u * rp, dh);
      one_round<kGeneral>(T, pos.z, pos.w, P, tc, lane, 2u * rp + 1u, dh);
    }
    if (tc.track && lane == tc.cyo && dh != 0)
      atomicAdd(P.h00, (unsigned long long)(long long)dh);

    // Write back this tile's window and slide to the next one.
    const bool last = (t + 1u == P.run);
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq)
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq)
#pragma unroll
        for (uint32_t sg = 0; sg < 2; ++sg) {
          const uint32_t sh = shx[xq];
          const uint32_t low = (1u << sh) - 1u;
          const uint32_t Tv = T[yq][xq][sg], Mv = M[yq][xq][sg];
          const uint32_t wl = (Mv & low) | (Tv << sh);                    // word t (left)
          const uint32_t cn = (Mv & ~low) | __funnelshift_l(Tv, 0u, sh);  // word t+1 (right)
          uint32_t* pl = addr(xq, yq, sg, t);
          if (t == 0u && sh != 0u) {
            // left word shared with the run to the left: xor in our bits only
            const uint32_t cur = __ldcg(pl);
            const uint32_t delta = (wl ^ cur) & ~low;
            if (delta) atomicXor(pl, delta);
          } else {
            __stcg(pl, wl);
          }
          uint32_t* pr = addr(xq, yq, sg, t + 1u);
          if (last) {
            if (sh != 0u) {  // right word shared with the run to the right
              const uint32_t cur = __ldcg(pr);
              const uint32_t delta = (cn ^ cur) & low;
              if (delta) atomicXor(pr, delta);
            }
          } else {
            const uint32_t N = __ldcg(addr(xq, yq, sg, t + 2u));
            T[yq][xq][sg] = __funnelshift_r(cn, N, sh);
            M[yq][xq][sg] = (cn & low) | (N & ~low);
          }
        }
  }
}

__global__ void advance_kernel(uint64_t* t_dev, uint32_t n) { *t_dev += n; }

}  // namespace

cudaError_t launch_sweep(const SweepParams& P, uint32_t warps_per_cta, cudaStream_t st) {
  const uint64_t warps = (uint64_t)P.runs_x * P.nty;
  const uint32_t wpc = warps_per_cta ? warps_per_cta : 8u;
  const uint64_t blocks = (warps + wpc - 1) / wpc;
  const bool general = !(P.Tp == 65536u && P.Tq == 0u);
  if (general)
    sweep_kernel<true><<<(unsigned)blocks, wpc * 32u, 0, st>>>(P);
  else
    sweep_kernel<false><<<(unsigned)blocks, wpc * 32u, 0, st>>>(P);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_advance(uint64_t* t_dev, uint32_t n, cudaStream_t st) {
  advance_kernel<<<1, 1, 0, st>>>(t_dev, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kpz
