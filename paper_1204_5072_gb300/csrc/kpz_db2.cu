// kpz_db2.cu -- one sweep with dead borders at both layers (the paper's
// earlier KPZ scheme, arXiv:1204.5072 Sec. 3.1: the dead-border decomposition
// of Sec. 3 used at the device layer and at the work-group layer).
//
// Device layer: the dead-border tiles of the main sweep (128 x 128 sites,
// origin redrawn every sweep, low row and column dead). Work-group layer: 16
// rounds per sweep; in round r the tile is cut into 4 x 4 blocks anchored at
// a random offset (dx, dy) that wraps inside the tile, each block's low row
// and column are its dead border, and each block makes one attempt at a
// uniformly random site of its 3 x 3 interior (n = floor(9 w / 2^32) from a
// Philox word w), accepted when a 16-bit Philox number is below Tp (minimum)
// or Tq (maximum), eq. (rule). Every site then has one attempt per sweep on
// average, and no two attempts of a round touch each other's sites, so the
// threads of a round need no ordering. The random streams (tags 9, 10, 11)
// are those of the oracle's orc_sweep_db2.
//
// This variant serves the comparison of decompositions, not speed: one CTA
// per tile holds the tile's window (plus the halo column and row of the
// neighbouring tiles' dead borders) as one byte per site in shared memory --
// bit 0 the height bit b of kpz_common.cuh, bit 1 its value at the start of
// the sweep -- and writes the changed sites back as XOR deltas (a storage
// word is shared with the neighbouring tiles, which change other bits of it).
#include "kpz_internal.h"

namespace kpz {
namespace {

constexpr uint32_t kWin = kTile + 1;          // window edge including the halo
constexpr uint32_t kThreads = 256;            // 4 blocks of 4 x 4 sites per thread
constexpr uint32_t kTagDbOff = 9u, kTagDbSite = 10u, kTagDbAcc = 11u;

__device__ __forceinline__ size_t site_word(const Geometry& g, uint32_t x, uint32_t y) {
  return g.word(x >> 7, plane(y & 3u, x & 3u), y >> 2);
}

__global__ void __launch_bounds__(kThreads) db2_kernel(const SweepParams P) {
  __shared__ uint8_t win[kWin][kWin];   // [v][u], u, v = 128: the neighbours' dead borders
  __shared__ int dh_tile;
  const uint32_t L = P.g.L, m = L - 1u;
  const uint32_t s = (uint32_t)(*P.t_dev) + P.s_add;
  const uint4 o = philox(kTagOrigin << 28, 0u, s, P.sample, P.k0, P.k1);
  const uint32_t T = blockIdx.x, tx = T % P.ntx, ty = T / P.ntx;
  const uint32_t x0 = (o.x + tx * kTile) & m, y0 = (o.y + ty * kTile) & m;
  if (threadIdx.x == 0) dh_tile = 0;
  for (uint32_t idx = threadIdx.x; idx < kWin * kWin; idx += kThreads) {
    const uint32_t u = idx % kWin, v = idx / kWin, x = (x0 + u) & m, y = (y0 + v) & m;
    const uint32_t b = (__ldcg(P.lat + site_word(P.g, x, y)) >> ((x >> 2) & 31u)) & 1u;
    win[v][u] = (uint8_t)(b | (b << 1));
  }
  __syncthreads();
  const uint32_t par0 = (x0 + y0 + P.g.par) & 1u;    // parity of local site (0, 0)
  const uint4 S = philox(kTagDbOff << 28, T, s, P.sample, P.k0, P.k1);
  int dh = 0;
  for (uint32_t r = 0; r < kRounds; ++r) {
    const uint32_t Sw = r < 8u ? S.x : S.y;
    const uint32_t dx = (Sw >> (4u * (r & 7u))) & 3u, dy = (Sw >> (4u * (r & 7u) + 2u)) & 3u;
    const uint4 w = philox((kTagDbSite << 28) | (r << 20) | threadIdx.x, T, s, P.sample, P.k0, P.k1);
    const uint4 a = philox((kTagDbAcc << 28) | (r << 20) | threadIdx.x, T, s, P.sample, P.k0, P.k1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w}, as[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (uint32_t j = 0; j < 4u; ++j) {
      const uint32_t k = 4u * threadIdx.x + j, kx = k % (kTile / 4u), ky = k / (kTile / 4u);
      const uint32_t n = __umulhi(ws[j], 9u);
      const uint32_t u = (dx + 4u * kx + 1u + n % 3u) & (kTile - 1u);
      const uint32_t v = (dy + 4u * ky + 1u + n / 3u) & (kTile - 1u);
      if (u == 0u || v == 0u) continue;                      // the tile's dead border
      const uint32_t bs = win[v][u] & 1u;
      const uint32_t hp = (par0 + u + v) & 1u;               // neighbour higher iff b(n) ^ b(s) == hp
      const bool hl = ((win[v][u - 1] ^ bs) & 1u) == hp, hr = ((win[v][u + 1] ^ bs) & 1u) == hp;
      const bool hd = ((win[v - 1][u] ^ bs) & 1u) == hp, hu = ((win[v + 1][u] ^ bs) & 1u) == hp;
      const uint32_t U = as[j] >> 16;
      const bool is_min = hl && hr && hd && hu, is_max = !hl && !hr && !hd && !hu;
      if ((is_min && U < P.Tp) || (is_max && U < P.Tq)) {
        win[v][u] ^= 1u;
        if (((x0 + u) & m) == 0u && ((y0 + v) & m) == 0u) dh += is_min ? 2 : -2;
      }
    }
    __syncthreads();
  }
  if (dh) atomicAdd(&dh_tile, dh);
  for (uint32_t idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
    const uint32_t u = idx % kTile, v = idx / kTile;
    const uint32_t c = win[v][u];
    if ((c ^ (c >> 1)) & 1u) {
      const uint32_t x = (x0 + u) & m, y = (y0 + v) & m;
      atomicXor(P.lat + site_word(P.g, x, y), 1u << ((x >> 2) & 31u));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && dh_tile) atomicAdd(P.h00, (unsigned long long)(long long)dh_tile);
}

}  // namespace

cudaError_t launch_sweep_db2(const SweepParams& P, cudaStream_t st) {
  if (P.nty != P.ntx || P.g.L / P.ntx != kTile) return cudaErrorInvalidValue;
  db2_kernel<<<P.ntx * P.nty, kThreads, 0, st>>>(P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kpz
