// kpz_w2.cuh -- exact W^2 building blocks shared by the single-lattice
// roughness kernel (kpz_observe.cu) and the ensemble kernel's W^2 bands
// (kpz_batch.cu): eq. (Wdef) with the heights of the gauge h(0,0) = 0.
//
// Along a row, h(i+1, j) = h(i, j) + sigma_x(i, j) with sigma_x = +-1 read from
// the height bits (kpz_common.cuh). A 128-site block of a row is cut into 16
// runs of 8 consecutive sites; for each run a table gives, from its 8 step
// bits, the height change D and the sums A1 = sum r, A2 = sum r^2 of the
// heights r relative to its first site, so a run starting at height h adds
// 8h + A1 to S1 and 8h^2 + 2h A1 + A2 to S2.
//
// Run bytes: bits (0, 1) = steps of plane 0 at cells c, c+1, bits (2, 3)
// plane 1, (4, 5) plane 2, (6, 7) plane 3; in x order the sites are bits
// 0, 2, 4, 6, 1, 3, 5, 7.
#pragma once
#include "kpz_common.cuh"

namespace kpz {
namespace w2 {

__device__ __forceinline__ uint32_t parity_mask(uint32_t v) { return (v & 1u) ? ~0u : 0u; }

// sigma_x planes of one 128-site block of row j: bit c of S[x4] is 1 when
// sigma_x(128K + 4c + x4, j) = +1. P = bit planes of the block, nxt = bit of
// site 128K + 128.
__device__ __forceinline__ void sigma_x_planes(const uint32_t (&P)[4], uint32_t nxt, uint32_t j,
                                               uint32_t par, uint32_t (&S)[4]) {
#pragma unroll
  for (uint32_t x4 = 0; x4 < 4; ++x4) {
    const uint32_t right = (x4 < 3) ? P[x4 < 3 ? x4 + 1 : 0] : ((P[0] >> 1) | (nxt << 31));
    S[x4] = ~(right ^ P[x4] ^ parity_mask(x4 + j + par));
  }
}

// Exact S1 = sum h and S2 = sum h^2 (eq. Wdef). Lane <-> row j = 4R + y4 with
// consecutive R per warp (coalesced plane loads). A 128-site block is cut into
// 16 runs of 8 consecutive sites; for each run a table gives, from its 8 step
// bits, the height change D and the sums A1 = sum r, A2 = sum r^2 of the
// heights r relative to its first site, so a run starting at height h adds
// 8h + A1 to S1 and 8h^2 + 2h A1 + A2 to S2. Sums are relative to the block's
// first site in 32-bit, then promoted to 64-bit.
//
// Run bytes: bits (0, 1) = steps of sites 4c and 4c+4 of plane 0 at cells
// c, c+1, bits (2, 3) plane 1, (4, 5) plane 2, (6, 7) plane 3; in x order the
// sites are bits 0, 2, 4, 6, 1, 3, 5, 7.
constexpr uint32_t kRunTable = 256;
constexpr uint32_t kRunTableWords = kRunTable * 32;   // one copy per lane

// Table entry of run byte b: A2 | (A1 + 28) << 8 | (D + 8) << 16.
__device__ __forceinline__ uint32_t run_entry(uint32_t b) {
  int32_t r = 0, a1 = 0, a2 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t bit = (b >> ((k & 3) * 2 + (k >> 2))) & 1u;
    a1 += r;
    a2 += r * r;
    r += 2 * (int32_t)bit - 1;
  }
  return (uint32_t)a2 | ((uint32_t)(a1 + 28) << 8) | ((uint32_t)(r + 8) << 16);
}

// The 16 run bytes of a block from its step planes S: u[q] byte m holds the
// run of cells 8m + 2q' .. 8m + 2q' + 1 with q' = (0, 2, 1, 3)[q].
__device__ __forceinline__ void run_bytes(const uint32_t (&S)[4], uint32_t (&u)[4]) {
  const uint32_t t01 = (S[0] & 0x33333333u) | ((S[1] << 2) & 0xCCCCCCCCu);   // cells 4k, 4k+1
  const uint32_t t01b = ((S[0] >> 2) & 0x33333333u) | (S[1] & 0xCCCCCCCCu);  // cells 4k+2, 4k+3
  const uint32_t t23 = (S[2] & 0x33333333u) | ((S[3] << 2) & 0xCCCCCCCCu);
  const uint32_t t23b = ((S[2] >> 2) & 0x33333333u) | (S[3] & 0xCCCCCCCCu);
  u[0] = (t01 & 0x0F0F0F0Fu) | ((t23 << 4) & 0xF0F0F0F0u);    // cells 8m, 8m+1
  u[1] = (t01b & 0x0F0F0F0Fu) | ((t23b << 4) & 0xF0F0F0F0u);  // cells 8m+2, 8m+3
  u[2] = ((t01 >> 4) & 0x0F0F0F0Fu) | (t23 & 0xF0F0F0F0u);    // cells 8m+4, 8m+5
  u[3] = ((t01b >> 4) & 0x0F0F0F0Fu) | (t23b & 0xF0F0F0F0u);  // cells 8m+6, 8m+7
}

// Fill the run table, one copy per lane (entry e of lane l at e*32 + l: no
// bank conflicts); all threads of the block take part, then synchronise.
__device__ __forceinline__ void fill_run_table(uint32_t* tab) {
  for (uint32_t e = threadIdx.x; e < kRunTable; e += blockDim.x) {
    const uint32_t v = run_entry(e);
#pragma unroll 8
    for (uint32_t l = 0; l < 32; ++l) tab[e * 32u + l] = v;
  }
  __syncthreads();
}

// Height change h and relative sums a1, a2 of one 128-site block with step
// planes S, from the lane's copy tl = tab + lane.
__device__ __forceinline__ void block_sums(const uint32_t* tl, const uint32_t (&S)[4], int32_t& h,
                                           int32_t& a1, int32_t& a2) {
  uint32_t u[4];
  run_bytes(S, u);
  h = 0; a1 = 0; a2 = 0;
#pragma unroll
  for (uint32_t m = 0; m < 4; ++m)
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t w = tl[((u[q] >> (8u * m)) & 0xFFu) * 32u];
      const int32_t A2 = (int32_t)(w & 0xFFu), A1 = (int32_t)((w >> 8) & 0xFFu) - 28;
      a1 += 8 * h + A1;
      a2 += h * (8 * h + 2 * A1) + A2;
      h += (int32_t)(w >> 16) - 8;
    }
}

}  // namespace w2
}  // namespace kpz
