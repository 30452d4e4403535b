// kpz_rounds.cuh -- the 16 single-hit rounds of one tile of 128 x (128 CR)
// sites held by a warp in registers (arXiv:1204.5072, Sec. 3.1; update rule
// eq. rule, Sec. 2.1).
//
// Lane l holds cell rows CR*l .. CR*l + CR - 1 of the tile; T[r][y'][x'] holds
// the height bits of site (x', y') of the 4 x 4 cells of its r-th cell row
// (bit c = cell c). A round evaluates the rule for the four
// sites of the active quadrant on all 32 cells at once with bitwise logic: a
// neighbour is higher iff its bit equals v = b(s) ^ parity(s); a minimum has
// all four neighbours equal to v, a maximum none; a move toggles b(s).
// Neighbours in x come from a 1-bit shift (cells c-1, c+1), neighbours in y
// from the lane's other cell row or the lanes above and below (warp
// shuffles); hx[r][y'] (bit 0) is the column right of the tile and hy[x']
// (lane 31) the row below it, both dead borders of neighbouring tiles that
// nobody changes during the sweep. Within a round each cell moves at most one
// site and no selected site is a neighbour of another selected site, so the
// order in which cells and cell rows are evaluated does not matter.
#pragma once
#include "kpz_internal.h"

namespace kpz {
namespace rounds {

constexpr uint32_t kFull = 0xffffffffu;

// Philox draw of a tile: from the round keys in shared memory (tc.rk) or,
// without kSK, by advancing the key (P.k0, P.k1).
struct TileCtx;
template <bool kSK>
__device__ __forceinline__ uint4 draw(const SweepParams& P, const TileCtx& tc, uint32_t c0);

struct TileCtx {
  uint32_t tid;           // tile id ty*ntx + tx (Philox counter word 1)
  uint32_t s;             // sweep index (Philox counter word 2)
  uint32_t setw;          // 16 x 2 bits: quadrant set of each round
  uint32_t first_row_ok;  // ~0 unless lane 0 (tile row v = 0 is dead)
  bool last_lane;         // lane 31: the row below comes from the halo
  bool track;             // this tile contains site (0,0)
  uint32_t xo, yo, co, cyo;  // site (0,0): column, row in the cell, cell, cell row
  const uint4* rk;        // round keys in shared memory (kSK)
  uint32_t pm;            // all ones when the tile's site (0,0) is odd (run-time parity)
  // Tiles without a dead border (kLive, one cell row per lane): bit 0 of
  // hxl[y'] is the site left of the tile in row y' of the lane's cell row;
  // hyu[x'] (lane 0) the row above the tile, cells as in T.
  uint32_t hxl[4], hyu[4];
};

template <bool kSK>
__device__ __forceinline__ uint4 draw(const SweepParams& P, const TileCtx& tc, uint32_t c0) {
  if (kSK) return philox_sk(c0, tc.tid, tc.s, P.sample, tc.rk);
  return philox(c0, tc.tid, tc.s, P.sample, P.k0, P.k1);
}

// Bit-serial comparison U < T for the 32 cells of a cell row (U uniform
// 16-bit, level n = bit 15-n of U taken from bit c of word n&3 of Philox call
// n>>2, call m at counter word 0 = base | m; base holds the stream's tag). Only cells in needp (selected site is a minimum) and needq (a
// maximum) need a decision; a cell is decided at the first level where U and
// T differ, so the warp stops drawing levels once no cell of any lane is still
// tied. The outcome equals the full 16-level comparison. Used by the C = 2
// work-group layer and the colour-class reference; the 4 x 4 single-hit
// rounds draw only as deep as a tie needs (deep_accept below).
template <bool kSK>
__device__ __forceinline__ void acceptance(const SweepParams& P, const TileCtx& tc, uint32_t base,
                                           uint32_t needp, uint32_t needq, uint32_t& AP, uint32_t& AQ) {
  uint32_t ltp = 0u, ltq = 0u;
  uint32_t undp = (P.Tp == 0u || (P.Tp >> 16)) ? 0u : needp;
  uint32_t undq = (P.Tq == 0u || (P.Tq >> 16)) ? 0u : needq;
#pragma unroll 1
  for (uint32_t m = 0; m < 4; ++m) {
    if (4u * m >= P.nlev || !__any_sync(0xffffffffu, (undp | undq) != 0u)) break;
    const uint4 A = draw<kSK>(P, tc, base | m);
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

// Low twelve bits of the acceptance numbers of the tied candidates of one
// cell row in round r (eq. rule): tp / tq mark the minima / maxima whose top
// four bits equal their threshold's. The k-th tied cell (k = 0, 1, ... in
// increasing cell index) takes 16-bit half 4 (r & 1) + k of the round pair's
// deep block D for k < 4, and half (k - 4) mod 8 of overflow block
// 1 + (k - 4) / 8 of this round otherwise (half 2i = low, 2i + 1 = high 16
// bits of word i); it is accepted when those twelve bits are below its
// threshold's. Returns the accepted cells. A lane has about one tie in
// sixteen candidates: the first four are taken without branches, more (a
// few rounds in a hundred per warp) by a loop that draws the overflow blocks.
template <bool kSK>
__device__ __forceinline__ uint32_t deep_accept(const SweepParams& P, const TileCtx& tc, uint32_t rw, uint32_t r,
                                                uint32_t tp, uint32_t tq, const uint4& D) {
  const uint32_t wlo = (r & 1u) ? D.z : D.x, whi = (r & 1u) ? D.w : D.y;
  const uint32_t lp = P.Tp & 0xFFFu, lq = P.Tq & 0xFFFu;
  const uint32_t h[4] = {wlo & 0xFFFu, (wlo >> 16) & 0xFFFu, whi & 0xFFFu, (whi >> 16) & 0xFFFu};
  uint32_t m = tp | tq, acc = 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t bit = m & (0u - m);   // the k-th tied cell, 0 if there is none
    m ^= bit;
    acc |= (h[k] < ((bit & tq) ? lq : lp)) ? bit : 0u;
  }
  if (m != 0u) {
    uint4 X = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = 4u; m != 0u; ++k) {
      const uint32_t bit = m & (0u - m);
      m ^= bit;
      const uint32_t j = (k - 4u) & 7u;
      if (j == 0u) X = draw<kSK>(P, tc, (kTagDeep << 28) | (rw << 8) | (r << 3) | (1u + ((k - 4u) >> 3)));
      const uint32_t w = (j & 4u) ? ((j & 2u) ? X.w : X.z) : ((j & 2u) ? X.y : X.x);
      const uint32_t hk = ((j & 1u) ? (w >> 16) : w) & 0xFFFu;
      acc |= (hk < ((bit & tq) ? lq : lp)) ? bit : 0u;
    }
  }
  return acc;
}

// Neighbours of the active quadrant (QX, QY) that lie outside the cell (x)
// or outside the cell row (y): xn[r][d] for quadrant row y0 + d of cell row
// r, yn[r][d] for quadrant column x0 + d.
template <int QX, int QY, int CR, bool kLive>
__device__ __forceinline__ void quad_halo(const uint32_t (&T)[CR][4][4], const uint32_t (&hx)[CR][4],
                                          const uint32_t (&hy)[4], const TileCtx& tc,
                                          uint32_t (&xn)[CR][2], uint32_t (&yn)[CR][2]) {
  constexpr int x0 = 2 * QX, y0 = 2 * QY;
  // The one y-neighbour per column that lies in another lane.
  uint32_t ysh[2];
  if (QY == 0) {
    ysh[0] = __shfl_up_sync(kFull, T[CR - 1][3][x0], 1);
    ysh[1] = __shfl_up_sync(kFull, T[CR - 1][3][x0 + 1], 1);
    if (kLive && tc.first_row_ok == 0u) { ysh[0] = tc.hyu[x0]; ysh[1] = tc.hyu[x0 + 1]; }
  } else {
    const uint32_t d0 = __shfl_down_sync(kFull, T[0][0][x0], 1);
    const uint32_t d1 = __shfl_down_sync(kFull, T[0][0][x0 + 1], 1);
    ysh[0] = tc.last_lane ? hy[x0] : d0;
    ysh[1] = tc.last_lane ? hy[x0 + 1] : d1;
  }
#pragma unroll
  for (int row = 0; row < CR; ++row)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      xn[row][d] = (QX == 0) ? ((T[row][y0 + d][3] << 1) | (kLive ? tc.hxl[y0 + d] : 0u))  // cell c-1, col 3
                             : __funnelshift_r(T[row][y0 + d][0], hx[row][y0 + d], 1);     // cell c+1, col 0
      if (QY == 0) yn[row][d] = (row > 0) ? T[row > 0 ? row - 1 : 0][3][x0 + d] : ysh[d];
      else         yn[row][d] = (row < CR - 1) ? T[row < CR - 1 ? row + 1 : 0][0][x0 + d] : ysh[d];
    }
}

// The four neighbours of quadrant site (dx, dy) of cell row r and the bit v
// that marks a higher neighbour (v = b(s) ^ parity(s)). kPar = parity of the
// tile's site (0,0), or 2: taken at run time from tc.pm (all ones when odd).
template <int QX, int QY, int kPar, int CR>
struct SiteView {
  uint32_t s, nL, nR, nU, nD, v;
  __device__ __forceinline__ SiteView(const uint32_t (&T)[CR][4][4], const uint32_t (&xn)[CR][2],
                                      const uint32_t (&yn)[CR][2], const TileCtx& tc, int row, int dx,
                                      int dy) {
    const int xp = 2 * QX + dx, yp = 2 * QY + dy;
    s = T[row][yp][xp];
    nL = (xp > 0) ? T[row][yp][xp > 0 ? xp - 1 : 0] : xn[row][dy];
    nR = (xp < 3) ? T[row][yp][xp < 3 ? xp + 1 : 3] : xn[row][dy];
    nU = (yp > 0) ? T[row][yp > 0 ? yp - 1 : 0][xp] : yn[row][dx];
    nD = (yp < 3) ? T[row][yp < 3 ? yp + 1 : 3][xp] : yn[row][dx];
    if (kPar == 2) v = s ^ (((xp + yp) & 1) ? ~tc.pm : tc.pm);
    else           v = ((kPar + xp + yp) & 1) ? ~s : s;
  }
};

// Cells whose random site (Xi, Yi) is quadrant site (dx, dy), without the
// dead border (tile column u = 0 and row v = 0) unless kLive.
template <int QX, int QY, bool kLive>
__device__ __forceinline__ uint32_t selected(uint32_t Xi, uint32_t Yi, const TileCtx& tc, int row, int dx, int dy) {
  uint32_t sel = (dx ? Xi : ~Xi) & (dy ? Yi : ~Yi);
  if (!kLive) {
    if (QX == 0 && dx == 0) sel &= ~1u;
    if (QY == 0 && dy == 0 && row == 0) sel &= tc.first_row_ok;
  }
  return sel;
}

// Selected local minima (fmin) of one single-hit round with active quadrant
// (QX, QY), from the state before the round, for every cell row (the
// p = 1, q = 0 path). Xi[r], Yi[r]: position bits of cell row r. Selected
// sites are never neighbours of each other, so masks taken before any flip
// equal masks taken site by site.
template <int QX, int QY, int kPar, int CR, bool kLive = false>
__device__ __forceinline__ void quad_masks(const uint32_t (&T)[CR][4][4], const uint32_t (&Xi)[CR],
                                           const uint32_t (&Yi)[CR], const uint32_t (&hx)[CR][4],
                                           const uint32_t (&hy)[4], const TileCtx& tc,
                                           uint32_t (&fmin)[CR][2][2]) {
  uint32_t xn[CR][2], yn[CR][2];
  quad_halo<QX, QY, CR, kLive>(T, hx, hy, tc, xn, yn);
#pragma unroll
  for (int row = 0; row < CR; ++row)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const SiteView<QX, QY, kPar, CR> n(T, xn, yn, tc, row, dx, dy);
        fmin[row][dy][dx] = selected<QX, QY, kLive>(Xi[row], Yi[row], tc, row, dx, dy) &
                            ~(n.nL ^ n.v) & ~(n.nR ^ n.v) & ~(n.nU ^ n.v) & ~(n.nD ^ n.v);
      }
}

// Apply the moves of a p = 1, q = 0 round with active quadrant (QX, QY):
// count those of site (0,0) when the tile holds it, then toggle the bits.
template <int QX, int QY, bool kTrack, int CR>
__device__ __forceinline__ void quad_flips(uint32_t (&T)[CR][4][4], const uint32_t (&fmin)[CR][2][2],
                                           const TileCtx& tc, uint32_t lane, int& dh) {
  constexpr int x0 = 2 * QX, y0 = 2 * QY;
#pragma unroll
  for (int row = 0; row < CR; ++row) {
    if (kTrack && CR * lane + row == tc.cyo) {
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
          if ((uint32_t)(x0 + dx) == tc.xo && (uint32_t)(y0 + dy) == tc.yo)
            dh += 2 * (int)((fmin[row][dy][dx] >> tc.co) & 1u);
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) T[row][y0 + dy][x0 + dx] ^= fmin[row][dy][dx];
  }
}

// Candidates of one general-rate round with active quadrant (QX, QY): the
// selected sites whose four neighbours are all higher (a local minimum) or
// all lower (a local maximum) -- all four neighbour bits equal, which does
// not depend on v. Per cell row, upc marks the cells whose candidate is a
// minimum, uqc those whose candidate is a maximum (a cell has at most one).
template <int QX, int QY, int kPar, int CR, bool kLive = false>
__device__ __forceinline__ void quad_cands(const uint32_t (&T)[CR][4][4], const uint32_t (&Xi)[CR],
                                           const uint32_t (&Yi)[CR], const uint32_t (&hx)[CR][4],
                                           const uint32_t (&hy)[4], const TileCtx& tc,
                                           uint32_t (&cand)[CR][2][2], uint32_t (&upc)[CR], uint32_t (&uqc)[CR]) {
  uint32_t xn[CR][2], yn[CR][2];
  quad_halo<QX, QY, CR, kLive>(T, hx, hy, tc, xn, yn);
#pragma unroll
  for (int row = 0; row < CR; ++row) {
    uint32_t mn = 0u, any = 0u;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const SiteView<QX, QY, kPar, CR> n(T, xn, yn, tc, row, dx, dy);
        const uint32_t c = selected<QX, QY, kLive>(Xi[row], Yi[row], tc, row, dx, dy) &
                           ~(n.nL ^ n.nR) & ~(n.nU ^ n.nD) & ~(n.nL ^ n.nU);
        cand[row][dy][dx] = c;
        mn |= c & ~(n.nL ^ n.v);
        any |= c;
      }
    upc[row] = mn;
    uqc[row] = any & ~mn;
  }
}

// Apply the accepted moves of a general-rate round: the candidates of the
// cells in acc toggle; site (0,0) counts +2 for a minimum, -2 for a maximum.
template <int QX, int QY, bool kTrack, int CR>
__device__ __forceinline__ void quad_flips_acc(uint32_t (&T)[CR][4][4], const uint32_t (&cand)[CR][2][2],
                                               const uint32_t (&acc)[CR], const uint32_t (&upc)[CR],
                                               const TileCtx& tc, uint32_t lane, int& dh) {
  constexpr int x0 = 2 * QX, y0 = 2 * QY;
#pragma unroll
  for (int row = 0; row < CR; ++row) {
    if (kTrack && CR * lane + row == tc.cyo) {
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
          if ((uint32_t)(x0 + dx) == tc.xo && (uint32_t)(y0 + dy) == tc.yo) {
            const uint32_t f = cand[row][dy][dx] & acc[row];
            dh += 2 * (int)(((f & upc[row]) >> tc.co) & 1u) - 2 * (int)(((f & ~upc[row]) >> tc.co) & 1u);
          }
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) T[row][y0 + dy][x0 + dx] ^= cand[row][dy][dx] & acc[row];
  }
}

// One single-hit round (Sec. 3.1): the quadrant set k of round r is uniform
// over the warp, so the round dispatches once on it. The p = 1, q = 0 path
// takes masks and flips in one branch; the general path takes the candidates
// in one branch, decides acceptance for all quadrants with the same code (one
// copy of the acceptance draws), then flips in a second branch.
// Acceptance (eq. rule, U < T with U uniform 16-bit): the top four bits of
// every candidate come bit-sliced from one Philox block per cell row and
// round; only candidates tied with their threshold there take low bits
// (deep_accept), from the deep block D of the round pair, drawn by the first
// round of the pair that has a tie in the warp (haveD).
template <bool kGeneral, int kPar, bool kTrack, int CR, bool kSK, bool kLive = false>
__device__ __forceinline__ void one_round(uint32_t (&T)[CR][4][4], const uint32_t (&Xi)[CR],
                                          const uint32_t (&Yi)[CR], const uint32_t (&hx)[CR][4],
                                          const uint32_t (&hy)[4], const SweepParams& P,
                                          const TileCtx& tc, uint32_t lane, uint32_t r, int& dh,
                                          uint4 (&D)[CR], bool& haveD) {
  const uint32_t k = (tc.setw >> (2u * r)) & 3u;
  if (!kGeneral) {
    uint32_t fmin[CR][2][2];
    switch (k) {
      case 0: quad_masks<0, 0, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, fmin);
              quad_flips<0, 0, kTrack, CR>(T, fmin, tc, lane, dh); break;
      case 1: quad_masks<1, 0, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, fmin);
              quad_flips<1, 0, kTrack, CR>(T, fmin, tc, lane, dh); break;
      case 2: quad_masks<0, 1, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, fmin);
              quad_flips<0, 1, kTrack, CR>(T, fmin, tc, lane, dh); break;
      default: quad_masks<1, 1, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, fmin);
               quad_flips<1, 1, kTrack, CR>(T, fmin, tc, lane, dh); break;
    }
    return;
  }
  uint32_t cand[CR][2][2], upc[CR], uqc[CR];
  switch (k) {
    case 0: quad_cands<0, 0, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, cand, upc, uqc); break;
    case 1: quad_cands<1, 0, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, cand, upc, uqc); break;
    case 2: quad_cands<0, 1, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, cand, upc, uqc); break;
    default: quad_cands<1, 1, kPar, CR, kLive>(T, Xi, Yi, hx, hy, tc, cand, upc, uqc); break;
  }
  uint32_t acc[CR];   // cells whose candidate moves
  if (kPar == 2) {
    // Run-time parity (the batched ensemble): one compare for minima and
    // maxima. b[n] is the threshold bit of each cell at level n (Tp's for a
    // minimum, Tq's for a maximum); U < T from the least significant of the
    // four levels up, lt = MAJ(~u, lt, b) per level, gives the cells decided
    // there, and the cells equal to their threshold on all four are the ties.
    const uint32_t dpm = (P.Tp != 0u && P.Tp < 65536u) ? ~0u : 0u;
    const uint32_t dqm = (P.Tq != 0u && P.Tq < 65536u) ? ~0u : 0u;
    const uint32_t pall = (P.Tp >> 16) ? ~0u : 0u, qall = (P.Tq >> 16) ? ~0u : 0u;
    uint32_t dm[CR], any = 0u;
#pragma unroll
    for (int row = 0; row < CR; ++row) {
      dm[row] = (upc[row] & dpm) | (uqc[row] & dqm);   // candidates that need random bits
      acc[row] = (upc[row] & pall) | (uqc[row] & qall);
      any |= dm[row];
    }
    if (__any_sync(kFull, any != 0u)) {
      uint32_t ties = 0u, tie[CR];
#pragma unroll
      for (int row = 0; row < CR; ++row) {
        const uint4 A = draw<kSK>(P, tc, (kTagAcc << 28) | ((CR * lane + row) << 4) | r);
        const uint32_t w[4] = {A.x, A.y, A.z, A.w};
        uint32_t b[4];
#pragma unroll
        for (uint32_t n = 0; n < 4u; ++n) {
          const uint32_t bp = 0u - ((P.Tp >> (15u - n)) & 1u);
          const uint32_t bq = 0u - ((P.Tq >> (15u - n)) & 1u);
          b[n] = (upc[row] & bp) | (~upc[row] & bq);
        }
        uint32_t lt = 0u;
#pragma unroll
        for (int n = 3; n >= 0; --n) lt = (~w[n] & lt) | (~w[n] & b[n]) | (lt & b[n]);
        uint32_t tq = dm[row];
#pragma unroll
        for (uint32_t n = 0; n < 4u; ++n) tq &= ~(w[n] ^ b[n]);
        acc[row] |= lt & dm[row];
        tie[row] = tq;
        ties |= tq;
      }
      if (__any_sync(kFull, ties != 0u)) {
        if (!haveD) {
#pragma unroll
          for (int row = 0; row < CR; ++row)
            D[row] = draw<kSK>(P, tc, (kTagDeep << 28) | ((CR * lane + row) << 8) | ((r & 14u) << 3));
          haveD = true;
        }
#pragma unroll
        for (int row = 0; row < CR; ++row)
          acc[row] |= deep_accept<kSK>(P, tc, CR * lane + row, r, tie[row] & upc[row], tie[row] & ~upc[row], D[row]);
      }
    }
  } else {
    // Fixed parity (single lattices): minima and maxima compared separately,
    // most significant level first (the faster form here).
    const bool drawp = P.Tp != 0u && P.Tp < 65536u, drawq = P.Tq != 0u && P.Tq < 65536u;
    uint32_t AP[CR], AQ[CR], up[CR], uq[CR];
    uint32_t any = 0u;
#pragma unroll
    for (int row = 0; row < CR; ++row) {
      AP[row] = (P.Tp >> 16) ? ~0u : 0u;
      AQ[row] = (P.Tq >> 16) ? ~0u : 0u;
      up[row] = drawp ? upc[row] : 0u;
      uq[row] = drawq ? uqc[row] : 0u;
      any |= up[row] | uq[row];
    }
    if (__any_sync(kFull, any != 0u)) {
      uint32_t ties = 0u;
#pragma unroll
      for (int row = 0; row < CR; ++row) {
        const uint4 A = draw<kSK>(P, tc, (kTagAcc << 28) | ((CR * lane + row) << 4) | r);
        const uint32_t w[4] = {A.x, A.y, A.z, A.w};
        uint32_t ltp = 0u, ltq = 0u;
#pragma unroll
        for (uint32_t n = 0; n < 4u; ++n) {   // levels 0..3: bits 15..12 of U and T
          const uint32_t bp = 0u - ((P.Tp >> (15u - n)) & 1u);
          const uint32_t bq = 0u - ((P.Tq >> (15u - n)) & 1u);
          ltp |= up[row] & ~w[n] & bp;
          up[row] &= ~(w[n] ^ bp);
          ltq |= uq[row] & ~w[n] & bq;
          uq[row] &= ~(w[n] ^ bq);
        }
        AP[row] |= ltp;
        AQ[row] |= ltq;
        ties |= up[row] | uq[row];
      }
      if (__any_sync(kFull, ties != 0u)) {
        if (!haveD) {
#pragma unroll
          for (int row = 0; row < CR; ++row)
            D[row] = draw<kSK>(P, tc, (kTagDeep << 28) | ((CR * lane + row) << 8) | ((r & 14u) << 3));
          haveD = true;
        }
#pragma unroll
        for (int row = 0; row < CR; ++row) {
          const uint32_t deep = deep_accept<kSK>(P, tc, CR * lane + row, r, up[row], uq[row], D[row]);
          AP[row] |= up[row] & deep;
          AQ[row] |= uq[row] & deep;
        }
      }
    }
#pragma unroll
    for (int row = 0; row < CR; ++row) acc[row] = (upc[row] & AP[row]) | (uqc[row] & AQ[row]);
  }
  switch (k) {
    case 0: quad_flips_acc<0, 0, kTrack, CR>(T, cand, acc, upc, tc, lane, dh); break;
    case 1: quad_flips_acc<1, 0, kTrack, CR>(T, cand, acc, upc, tc, lane, dh); break;
    case 2: quad_flips_acc<0, 1, kTrack, CR>(T, cand, acc, upc, tc, lane, dh); break;
    default: quad_flips_acc<1, 1, kTrack, CR>(T, cand, acc, upc, tc, lane, dh); break;
  }
}

// The 16 single-hit rounds of one tile, two rounds per Philox block of
// positions of each cell row (counter: cell row cy = CR*lane + r, round pair).
template <bool kGeneral, int kPar, bool kTrack, int CR, bool kSK, bool kLive = false>
__device__ __forceinline__ void tile_rounds(uint32_t (&T)[CR][4][4], const uint32_t (&hx)[CR][4],
                                            const uint32_t (&hy)[4], const SweepParams& P,
                                            const TileCtx& tc, uint32_t lane, int& dh) {
#pragma unroll 1
  for (uint32_t rp = 0; rp < kRounds / 2; ++rp) {
    uint32_t X0[CR], Y0[CR], X1[CR], Y1[CR];
#pragma unroll
    for (int row = 0; row < CR; ++row) {
      const uint4 pos = draw<kSK>(P, tc, (kTagPos << 28) | ((CR * lane + row) << 3) | rp);
      X0[row] = pos.x; Y0[row] = pos.y; X1[row] = pos.z; Y1[row] = pos.w;
    }
    uint4 D[CR];          // deep acceptance block of the round pair (general rates)
    bool haveD = false;
    one_round<kGeneral, kPar, kTrack, CR, kSK, kLive>(T, X0, Y0, hx, hy, P, tc, lane, 2u * rp, dh, D, haveD);
    one_round<kGeneral, kPar, kTrack, CR, kSK, kLive>(T, X1, Y1, hx, hy, P, tc, lane, 2u * rp + 1u, dh, D, haveD);
  }
}

// The C = 2 limit of the work-group layer (one cell row per lane): 2 x 2
// cells whose four 1 x 1 quadrants are the sets. In a round with set (QX, QY)
// every 2 x 2 cell attempts its site (QX, QY), i.e. the four sites
// (QX + 2i, QY + 2j) of every 4 x 4 storage cell, no two of them neighbours.
// No position draws; the acceptance numbers of site a = 2j + i of the storage
// cells of cell row `lane` in round r use counter base lane << 6 | r << 4 | a << 2.
template <int QX, int QY, bool kGeneral, int kPar, bool kTrack, bool kSK>
__device__ __forceinline__ void c2_round(uint32_t (&T)[4][4], const uint32_t (&hx)[4],
                                         const uint32_t (&hy)[4], const SweepParams& P,
                                         const TileCtx& tc, uint32_t lane, uint32_t r, int& dh) {
  uint32_t ysh[2];   // neighbour in another lane of column QX + 2i
  if (QY == 0) {
    ysh[0] = __shfl_up_sync(kFull, T[3][QX], 1);
    ysh[1] = __shfl_up_sync(kFull, T[3][QX + 2], 1);
  } else {
    const uint32_t d0 = __shfl_down_sync(kFull, T[0][QX], 1);
    const uint32_t d1 = __shfl_down_sync(kFull, T[0][QX + 2], 1);
    ysh[0] = tc.last_lane ? hy[QX] : d0;
    ysh[1] = tc.last_lane ? hy[QX + 2] : d1;
  }
  uint32_t fmin[2][2], fmax[2][2];   // [j][i]: site (QX + 2i, QY + 2j)
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int xp = QX + 2 * i, yp = QY + 2 * j;
      const uint32_t s = T[yp][xp];
      const uint32_t nL = (xp > 0) ? T[yp][xp > 0 ? xp - 1 : 0] : (T[yp][3] << 1);
      const uint32_t nR = (xp < 3) ? T[yp][xp < 3 ? xp + 1 : 3] : __funnelshift_r(T[yp][0], hx[yp], 1);
      const uint32_t nU = (yp > 0) ? T[yp > 0 ? yp - 1 : 0][xp] : ysh[i];
      const uint32_t nD = (yp < 3) ? T[yp < 3 ? yp + 1 : 3][xp] : ysh[i];
      uint32_t sel = ~0u;
      if (xp == 0) sel &= ~1u;                 // tile column u = 0
      if (yp == 0) sel &= tc.first_row_ok;     // tile row v = 0
      const uint32_t v = ((kPar + xp + yp) & 1) ? ~s : s;   // bit of a higher neighbour
      const uint32_t hL = ~(nL ^ v), hR = ~(nR ^ v), hU = ~(nU ^ v), hD = ~(nD ^ v);
      fmin[j][i] = sel & hL & hR & hU & hD;
      fmax[j][i] = kGeneral ? (sel & ~hL & ~hR & ~hU & ~hD) : 0u;
    }
  if (kGeneral) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        uint32_t AP, AQ;
        acceptance<kSK>(P, tc, (kTagAcc << 28) | (lane << 6) | (r << 4) | (uint32_t)((2 * j + i) << 2), fmin[j][i],
                        fmax[j][i], AP, AQ);
        fmin[j][i] &= AP;
        fmax[j][i] &= AQ;
      }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int xp = QX + 2 * i, yp = QY + 2 * j;
      if (kTrack && lane == tc.cyo && (uint32_t)xp == tc.xo && (uint32_t)yp == tc.yo)
        dh += 2 * (int)((fmin[j][i] >> tc.co) & 1u) - 2 * (int)((fmax[j][i] >> tc.co) & 1u);
      T[yp][xp] ^= fmin[j][i] | fmax[j][i];
    }
}

// The four C = 2 rounds of one tile (sets from tc.setw, two bits per round).
template <bool kGeneral, int kPar, bool kTrack, bool kSK>
__device__ __forceinline__ void tile_rounds_c2(uint32_t (&T)[4][4], const uint32_t (&hx)[4],
                                               const uint32_t (&hy)[4], const SweepParams& P,
                                               const TileCtx& tc, uint32_t lane, int& dh) {
#pragma unroll 1
  for (uint32_t r = 0; r < 4u; ++r) {
    switch ((tc.setw >> (2u * r)) & 3u) {
      case 0: c2_round<0, 0, kGeneral, kPar, kTrack, kSK>(T, hx, hy, P, tc, lane, r, dh); break;
      case 1: c2_round<1, 0, kGeneral, kPar, kTrack, kSK>(T, hx, hy, P, tc, lane, r, dh); break;
      case 2: c2_round<0, 1, kGeneral, kPar, kTrack, kSK>(T, hx, hy, P, tc, lane, r, dh); break;
      default: c2_round<1, 1, kGeneral, kPar, kTrack, kSK>(T, hx, hy, P, tc, lane, r, dh); break;
    }
  }
}

}  // namespace rounds
}  // namespace kpz
