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
// Mapping: one warp owns a tile of 128 x 128 CR sites (a run of `run` tiles
// along x, processed in turn); lane l owns cell rows CR l .. CR l + CR - 1
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
// Scheduling: one wave of resident warps takes runs of P.run tiles from a
// work queue, so the sweep has no partial last wave and faster SMs take more
// runs. The words a run shares with its neighbours at either end are written
// back as XOR deltas against the tile's start copy, so no run reads memory
// that another run may be changing. On the p = 1, q = 0 path the Philox round
// keys are read from shared memory instead of being advanced per draw.
#include <algorithm>
#include <mutex>

#include "kpz_rounds.cuh"

namespace kpz {
namespace {

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
// M: per cell row and plane, the bits of the window's two block columns that
// lie outside the window; Pf: next block column, double-buffered; Hf: lane
// 31's halo row, a ring of three block columns.
template <int CR>
struct WarpStage {
  uint32_t M[CR][kPlanes][32];
  uint32_t Pf[2][CR][kPlanes][32];
  uint32_t Hf[3][4];
};
constexpr uint32_t kMaxWarpsPerCta = 8;

// One run: tiles tx0 .. tx0 + n - 1 of tile row ty (n <= ntx), left to right.
template <bool kGeneral, int CR>
__device__ __forceinline__ void sweep_run(const SweepParams& P, WarpStage<CR>& ws, const uint4* rk,
                                          uint32_t lane,
                                          uint32_t s, uint32_t ox, uint32_t oy, uint32_t ty,
                                          uint32_t tx0, uint32_t n) {
  constexpr uint32_t kTileY = kTile * CR;
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
  tc.last_lane = last_lane;
  const uint32_t vo = (0u - Y0) & (L - 1u);

  // Quadrant sets: on the p = 1 path lane l draws the set of tile t0 + l
  // (t0 = t & ~31) and the warp broadcasts it, one draw per 32 tiles.
  uint32_t set_lane = 0;
#pragma unroll 1
  for (uint32_t t = 0; t < n; ++t) {
    if (kGeneral) {
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
      for (uint32_t yq = 0; yq < 4; ++yq) hx[r][yq] = (ws.M[r][yq * 4][lane] >> shx[0]) & 1u;
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
    if (tc.track) {
      if (par) tile_rounds<kGeneral, 1, true, CR, !kGeneral>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, true, CR, !kGeneral>(T, hx, hy, P, tc, lane, dh);
    } else {
      if (par) tile_rounds<kGeneral, 1, false, CR, !kGeneral>(T, hx, hy, P, tc, lane, dh);
      else     tile_rounds<kGeneral, 0, false, CR, !kGeneral>(T, hx, hy, P, tc, lane, dh);
    }
    if (tc.track && lane == tc.cyo / CR && dh != 0)
      atomicAdd(P.h00, (unsigned long long)(long long)dh);

    // Write back block column t and slide the window to tile t+1.
    cp_async_wait();
    if (!kGeneral && CR == 1 && t != 0u && !last) {
      // Interior tile: both words of each window row are this run's alone.
#pragma unroll
      for (uint32_t xq = 0; xq < 4; ++xq) {
        const uint32_t sh = shx[xq];
        const uint32_t low = (1u << sh) - 1u;
        uint32_t* cl = col(xq, t);
#pragma unroll
        for (int r = 0; r < CR; ++r)
#pragma unroll
          for (uint32_t yq = 0; yq < 4; ++yq) {
            const uint32_t Tv = T[r][yq][xq], Mv = ws.M[r][yq * 4 + xq][lane];
            __stcg(cl + offY[r][yq], (Mv & low) | (Tv << sh));                // word t
            const uint32_t cn = (Mv & ~low) | __funnelshift_l(Tv, 0u, sh);    // word t+1
            const uint32_t N = ws.Pf[t & 1u][r][yq * 4 + xq][lane];           // block column t+2
            T[r][yq][xq] = __funnelshift_r(cn, N, sh);
            ws.M[r][yq * 4 + xq][lane] = (cn & low) | (N & ~low);
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
              ws.M[r][yq * 4 + xq][lane] = (cn & low) | (N & ~low);
            }
          }
      }
    }
    if (t + 2u < n) prefetch(t + 3u);   // for the end of tile t+1
  }
}

// Persistent sweep: the resident warps take chunks of P.run tiles of one
// tile row from a work queue (row-major order, one atomic per chunk, fetched
// a chunk ahead), so faster SMs take more chunks and the tail is one chunk.
// Every warp makes exactly one fetch past the last chunk; the warp whose
// fetch is the last of all (nchunks + W - 1) returns the counter to zero for
// the next launch.
template <bool kGeneral, int CR>
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
    sweep_run<kGeneral, CR>(P, ws, rk, lane, s, ox, oy, ty, (c - ty * cpr) * P.run, P.run);
    c = __shfl_sync(kFull, next, 0);
  }
  if (lane == 0 && c == nchunks + W - 1u) atomicExch(P.queue, 0u);
}

// Resident CTAs per SM of one sweep kernel at wpc warps per CTA (cached per device).
template <bool kGeneral, int CR>
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
  e = cudaFuncSetAttribute(sweep_kernel<kGeneral, CR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<kGeneral, CR>, (int)(wpc * 32u),
                                                    wpc * sizeof(WarpStage<CR>));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  ctas = (uint32_t)(per_sm > 0 ? per_sm : 1) * (uint32_t)(sms > 0 ? sms : 1);
  if (dev < kMaxDev) cache[dev][wpc] = ctas;
  return cudaSuccess;
}

template <bool kGeneral, int CR>
cudaError_t launch_cr(const SweepParams& P, uint32_t wpc, cudaStream_t st) {
  uint32_t ctas = 0;
  cudaError_t e = resident_ctas<kGeneral, CR>(wpc, ctas);
  if (e != cudaSuccess) return e;
  // One wave of resident warps, fewer if there are fewer tiles than warps.
  const uint64_t tiles = (uint64_t)P.ntx * P.nty;
  const uint64_t blocks = std::min<uint64_t>(ctas, (tiles + wpc - 1) / wpc);
  sweep_kernel<kGeneral, CR><<<(unsigned)blocks, wpc * 32u, wpc * sizeof(WarpStage<CR>), st>>>(P);
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
  if (tile_y == kTile)
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
