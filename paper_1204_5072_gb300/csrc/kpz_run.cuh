// kpz_run.cuh -- one run of tiles of one sweep, the unit of work of both the
// single-lattice sweep kernel (kpz_sweep.cu) and the ensemble kernel
// (kpz_batch.cu).
//
// Decomposition (arXiv:1204.5072, Sec. 3 and 3.1):
//   device layer     -- 128 x (128 CR) tiles whose grid origin (ox, oy) is
//                       redrawn every sweep; the low-x column and low-y row of a
//                       tile (its dead border) are never updated, so tiles do
//                       not interact and run concurrently;
//   work-group layer -- single-hit double tiling: each tile is split into
//                       4 x 4 cells, each cell into four 2 x 2 quadrants; in
//                       each of 16 rounds one random quadrant set is active
//                       and every cell makes one attempt at a random site of
//                       its active quadrant (kpz_rounds.cuh).
//
// Mapping: one warp owns a tile of 128 x 128 CR sites (a run of tiles along
// x, processed in turn); lane l owns cell rows CR l .. CR l + CR - 1
// (tile rows 4 CR l .. 4 CR l + 4 CR - 1). The tile lives in 16 CR registers
// per lane, one per site (x', y') of the 4 x 4 cell and cell row, bit c =
// cell c of the row. A round evaluates the rule for the four sites of the
// active quadrant on all 32 cells of a row at once with bitwise logic;
// neighbours in x come from a 1-bit shift (cells c-1, c+1), neighbours in y
// from the lane's other cell row or the lanes above and below (warp
// shuffles). The right neighbour of the last cell column and the row below
// the last lane belong to the next tiles' dead borders, which no one changes
// during the sweep: they are read once as halos. The next block column is
// copied into shared memory (cp.async) one tile ahead.
//
// A run is tiles tx0 .. tx0 + n - 1 of one tile row, swept left to right with a
// sliding two-word window per plane. The words a run shares with the runs to
// its left and right are written back as XOR deltas against the tile's start
// copy, so a run never reads memory another run may be changing. With kSK the
// Philox round keys come from shared memory (rk) and each lane draws the
// quadrant sets of a different tile. With kRtPar the tile parity is a run-time
// value, so one copy of the round code serves every tile (callers whose
// warps work on tiles of both parities at once).
#pragma once
#include "kpz_rounds.cuh"

namespace kpz {
namespace run {

using rounds::TileCtx;
using rounds::kFull;
using rounds::tile_rounds;

// Asynchronous 4-byte global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async4(uint32_t* smem, const uint32_t* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// The same copy, issued only where pred holds (no branch).
__device__ __forceinline__ void cp_async4_if(bool pred, uint32_t* smem, const uint32_t* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %0, 0;\n @p cp.async.ca.shared.global [%1], [%2], 4;\n}\n" ::"r"(
          (uint32_t)pred),
      "r"(sa), "l"(gmem)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Per-warp staging in shared memory (each lane only touches its own column):
// M: per cell row and plane, for the first tile the bits of block columns 0
// and 1 that lie outside its window, from then on the carry: the low shx bits
// of the next word to store (the top of the window just swept); Pf: block
// columns, double-buffered (while tile t is swept, Pf[(t+1)&1] holds block
// column t+1 as read and Pf[t&1] receives t+2); Hf: lane 31's halo row, a
// ring of three block columns.
template <int CR>
struct WarpStage {
  uint32_t M[CR][kPlanes][32];
  uint32_t Pf[2][CR][kPlanes][32];
  uint32_t Hf[3][4];
};
constexpr uint32_t kMaxWarpsPerCta = 8;

// One run: tiles tx0 .. tx0 + n - 1 of tile row ty (n <= ntx), left to right.
template <bool kGeneral, int CR, bool kSK, bool kRtPar = false, bool kC2 = false>
__device__ __forceinline__ void sweep_run(const SweepParams& P, WarpStage<CR>& ws, const uint4* rk,
                                          uint32_t lane,
                                          uint32_t s, uint32_t ox, uint32_t oy, uint32_t ty,
                                          uint32_t tx0, uint32_t n) {
  constexpr uint32_t kTileY = kTile * CR;
  static_assert(!kC2 || CR == 1, "the C = 2 work-group layer holds one cell row per lane");
  const uint32_t L = P.g.L, NR = P.g.NR, NB = P.g.NB;
  // Rows: tile row y' of this lane's cell row r lives in storage cell row
  // Rb + CR lane + r (+1 past a plane wrap), plane row (by+y')%4.
  const uint32_t Y0 = (oy + ty * kTileY) & (L - 1u);
  const uint32_t by = Y0 & 3u, Rb = Y0 >> 2;
  uint32_t offY[CR][4];
#pragma unroll
  for (int r = 0; r < CR; ++r)
#pragma unroll
    for (uint32_t yq = 0; yq < 4; ++yq)
      offY[r][yq] = ((by + yq) & 3u) * 4u * NR + ((Rb + CR * lane + r + ((by + yq) >> 2)) & (NR - 1u));
  const uint32_t offH = by * 4u * NR + ((Rb + 32u * CR) & (NR - 1u));  // row below the tile
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
      for (int r = 0; r < CR; ++r)
#pragma unroll
        for (uint32_t yq = 0; yq < 4; ++yq)
          cp_async4(&ws.Pf[t & 1u][r][yq * 4 + xq][lane], c + offY[r][yq]);
      cp_async4_if(last_lane, &ws.Hf[t % 3u][xq], c + offH);
    }
    cp_async_commit();
  };

  uint32_t T[CR][4][4];
  // Prologue: window of the first tile (block columns 0 and 1).
#pragma unroll
  for (uint32_t xq = 0; xq < 4; ++xq) {
    const uint32_t* c0 = col(xq, 0);
    const uint32_t* c1 = col(xq, 1);
    const uint32_t low = (1u << shx[xq]) - 1u;
#pragma unroll
    for (int r = 0; r < CR; ++r)
#pragma unroll
      for (uint32_t yq = 0; yq < 4; ++yq) {
        const uint32_t C = __ldcg(c0 + offY[r][yq]);
        const uint32_t N = __ldcg(c1 + offY[r][yq]);
        T[r][yq][xq] = __funnelshift_r(C, N, shx[xq]);
        ws.M[r][yq * 4 + xq][lane] = (C & low) | (N & ~low);
      }
    if (last_lane) {
      ws.Hf[0][xq] = __ldcg(c0 + offH);
      ws.Hf[1][xq] = __ldcg(c1 + offH);
    }
  }
  // Copy of the tile at its start, for the bits of the edge words that the
  // runs on either side share (written back as XOR deltas): tile 0's copy in
  // Pf[1], the last tile's in Pf[(n-1) & 1]; neither slot is in use then.
#pragma unroll
  for (int r = 0; r < CR; ++r)
#pragma unroll
    for (uint32_t p = 0; p < kPlanes; ++p) ws.Pf[1][r][p][lane] = T[r][p >> 2][p & 3u];
  if (n > 1u) prefetch(2u);

  TileCtx tc;
  tc.rk = rk;
  tc.s = s;
  tc.first_row_ok = lane == 0u ? 0u : ~0u;
  tc.pm = par ? ~0u : 0u;
  tc.last_lane = last_lane;
  const uint32_t vo = (0u - Y0) & (L - 1u);

  // Quadrant sets: with round keys in shared memory (kSK) lane l draws the set
  // of tile t0 + l (t0 = t & ~31) and the warp broadcasts it, one draw per 32
  // tiles; otherwise every lane draws the set of each tile.
  uint32_t set_lane = 0;
#pragma unroll 1
  for (uint32_t t = 0; t < n; ++t) {
    if (!kSK) {
      tc.tid = ty * P.ntx + tx0 + t;
      tc.setw = philox(kTagSet << 28, tc.tid, s, P.sample, P.k0, P.k1).x;
    } else {
      if ((t & 31u) == 0u) {
        tc.tid = ty * P.ntx + tx0 + t + lane;
        set_lane = philox_sk(kTagSet << 28, tc.tid, s, P.sample, rk).x;
      }
      tc.tid = ty * P.ntx + tx0 + t;
      tc.setw = __shfl_sync(kFull, set_lane, t & 31u);
    }
    const uint32_t uo = (0u - ((X0 + t * kTile) & (L - 1u))) & (L - 1u);
    tc.track = (uo < kTile) && (vo < kTileY);
    tc.xo = uo & 3u; tc.co = uo >> 2; tc.yo = vo & 3u; tc.cyo = vo >> 2;

    // Halos: column u = 128 (tile t+1's dead column) and, for lane 31, row v = 128 CR.
    uint32_t hx[CR][4], hy[4];
#pragma unroll
    for (int r = 0; r < CR; ++r)
#pragma unroll
      for (uint32_t yq = 0; yq < 4; ++yq)   // bit 0 of window t+1 = bit shx[0] of block column t+1
        hx[r][yq] = ((t == 0u ? ws.M[r][yq * 4][lane] : ws.Pf[(t + 1u) & 1u][r][yq * 4][lane]) >> shx[0]) & 1u;
#pragma unroll
    for (uint32_t xq = 0; xq < 4; ++xq)
      hy[xq] = last_lane ? __funnelshift_r(ws.Hf[t % 3u][xq], ws.Hf[(t + 1u) % 3u][xq], shx[xq]) : 0u;

    const bool last = (t + 1u == n);
    const uint32_t keep = t == 0u ? 1u : (t & 1u);   // slot of the start copy
    if (last && t != 0u) {
#pragma unroll
      for (int r = 0; r < CR; ++r)
#pragma unroll
        for (uint32_t p = 0; p < kPlanes; ++p) ws.Pf[keep][r][p][lane] = T[r][p >> 2][p & 3u];
    }

    int dh = 0;
    // The one tile per sweep that holds site (0,0) also counts its moves.
    if (kC2) {      // C = 2 work-group layer (one cell row per lane)
      auto& T0 = reinterpret_cast<uint32_t(&)[4][4]>(T[0]);
      if (tc.track) {
        if (par) rounds::tile_rounds_c2<kGeneral, 1, true, kSK>(T0, hx[0], hy, P, tc, lane, dh);
        else     rounds::tile_rounds_c2<kGeneral, 0, true, kSK>(T0, hx[0], hy, P, tc, lane, dh);
      } else {
        if (par) rounds::tile_rounds_c2<kGeneral, 1, false, kSK>(T0, hx[0], hy, P, tc, lane, dh);
        else     rounds::tile_rounds_c2<kGeneral, 0, false, kSK>(T0, hx[0], hy, P, tc, lane, dh);
      }
    } else if (kRtPar) {   // one copy of the rounds for both parities (tc.pm)
      if (tc.track) tile_rounds<kGeneral, 2, true, CR, kSK>(T, hx, hy, P, tc, lane, dh);
      else          tile_rounds<kGeneral, 2, false, CR, kSK>(T, hx, hy, P, tc, lane, dh);
    } else if (tc.track) {
      if (par) tile_rounds<kGeneral, 1, true, CR, kSK>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, true, CR, kSK>(T, hx, hy, P, tc, lane, dh);
    } else {
      if (par) tile_rounds<kGeneral, 1, false, CR, kSK>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, false, CR, kSK>(T, hx, hy, P, tc, lane, dh);
    }
    if (tc.track && lane == tc.cyo / CR && dh != 0)
      atomicAdd(P.h00, (unsigned long long)(long long)dh);

    // Write back block column t and slide the window to tile t+1.
    cp_async_wait();
    if (t != 0u && !last) {
      // Interior tile: both words of each window row are this run's alone.
      // One wide multiply-add gives the word to store, carry | T << sh, and
      // the next carry, T >> (32 - sh) (exact: the carry is below 2^sh); the
      // next window comes from the raw block columns t+1 and t+2 in staging.
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq) {
        const uint32_t sh = shx[xq];
        const uint32_t mul = 1u << sh;
        uint32_t* cl = col(xq, t);
#pragma unroll
        for (int r = 0; r < CR; ++r)
#pragma unroll
          for (uint32_t yq = 0; yq < 4; ++yq) {
            const uint32_t pi = yq * 4 + xq;
            unsigned long long w;
            asm("mad.wide.u32 %0, %1, %2, %3;"
                : "=l"(w)
                : "r"(T[r][yq][xq]), "r"(mul), "l"((unsigned long long)ws.M[r][pi][lane]));
            __stcg(cl + offY[r][yq], (uint32_t)w);                                    // word t
            ws.M[r][pi][lane] = (uint32_t)(w >> 32);
            T[r][yq][xq] = __funnelshift_r(ws.Pf[(t + 1u) & 1u][r][pi][lane], ws.Pf[t & 1u][r][pi][lane], sh);
          }
      }
    } else {
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq) {
        const uint32_t sh = shx[xq];
        const uint32_t low = (1u << sh) - 1u;
        uint32_t* cl = col(xq, t);
        uint32_t* cr = col(xq, t + 1u);
#pragma unroll
        for (int r = 0; r < CR; ++r)
#pragma unroll
          for (uint32_t yq = 0; yq < 4; ++yq) {
            const uint32_t Tv = T[r][yq][xq], Mv = ws.M[r][yq * 4 + xq][lane];
            const uint32_t wl = (Mv & low) | (Tv << sh);                    // word t
            const uint32_t cn = (Mv & ~low) | __funnelshift_l(Tv, 0u, sh);  // word t+1
            uint32_t* pl = cl + offY[r][yq];
            if (t == 0u && sh != 0u) {
              // left word shared with the run to the left: xor in our changes only
              const uint32_t delta = (Tv ^ ws.Pf[1][r][yq * 4 + xq][lane]) << sh;
              if (delta) atomicXor(pl, delta);
            } else {
              __stcg(pl, wl);
            }
            if (last) {
              if (sh != 0u) {  // right word shared with the run to the right
                const uint32_t delta = __funnelshift_l(Tv ^ ws.Pf[keep][r][yq * 4 + xq][lane], 0u, sh);
                if (delta) atomicXor(cr + offY[r][yq], delta);
              }
            } else {
              const uint32_t N = ws.Pf[t & 1u][r][yq * 4 + xq][lane];  // block column t+2
              T[r][yq][xq] = __funnelshift_r(cn, N, sh);
              ws.M[r][yq * 4 + xq][lane] = cn & low;   // the carry into word t+1
            }
          }
      }
    }
    if (t + 2u < n) prefetch(t + 3u);   // for the end of tile t+1
  }
}

}  // namespace run
}  // namespace kpz
