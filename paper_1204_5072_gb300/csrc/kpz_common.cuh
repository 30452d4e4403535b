// kpz_common.cuh -- device-side building blocks shared by the engine's kernels.
//
// HBM layout of a lattice of lateral size L (bit-sliced cell rows):
//   storage cell = 4 x 4 sites; cell row R = sites with y in [4R, 4R+4), R < L/4;
//   block column K = 32 consecutive storage cells along x (128 sites), K < L/128;
//   plane p = (y%4 * 4 + x%4) * 2 + sigma, sigma 0 = slope in x, 1 = slope in y.
//   word(K, p, R) = lat[(K*32 + p) * (L/4) + R]; bit c of it is the sigma-slope
//   (1 = +1) of site (128K + 4c + x%4, 4R + y%4).
// Each word holds one slope bit of 32 cells, so one logic instruction updates
// 32 cells ("multi-spin coding" of the bit-coded cellular automaton the paper
// relies on, Sec. 5). Lanes of a warp read consecutive R: loads and stores of
// a warp cover 128 contiguous bytes. The layout holds 2 bits per site.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kpz {

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplications whose high halves are mixed
// with the other two words and a round key advanced by two Weyl constants.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
    const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
    const uint32_t n0 = hiB ^ c1 ^ k0;
    const uint32_t n2 = hiA ^ c3 ^ k1;
    c0 = n0; c1 = loB; c2 = n2; c3 = loA;
    k0 += kWeylA; k1 += kWeylB;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Stream tags of the Philox counter word 0 (tag << 28 | index).
enum : uint32_t { kTagOrigin = 0u, kTagSet = 1u, kTagPos = 2u, kTagAcc = 3u };

constexpr uint32_t kTile = 128;      // tile edge in sites (device layer)
constexpr uint32_t kRounds = 16;     // single-hit rounds per sweep = sites per cell

struct Geometry {
  uint32_t L;        // lateral size (power of two, >= 128)
  uint32_t NR;       // L/4 cell rows
  uint32_t NB;       // L/128 block columns
  __host__ __device__ size_t word(uint32_t K, uint32_t p, uint32_t R) const {
    return ((size_t)K * 32u + p) * NR + R;
  }
};

__host__ __device__ constexpr uint32_t plane(uint32_t y4, uint32_t x4, uint32_t sigma) {
  return (y4 * 4u + x4) * 2u + sigma;
}

}  // namespace kpz
