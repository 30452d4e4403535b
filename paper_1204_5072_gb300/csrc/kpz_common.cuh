// kpz_common.cuh -- device-side building blocks shared by the engine's kernels.
//
// State encoding. Every move changes a height by +-2 (eq. rule), so a site's
// height keeps the parity h(i,j) = i + j + par (mod 2) with par = h(0,0) mod 2
// of the start surface. Its height modulo 4 is therefore fixed by one bit,
//   b(i,j) = (h(i,j) >> 1) & 1,      h mod 4 = 2 b + (i + j + par) mod 2,
// and the octahedron slopes follow from neighbouring bits:
//   neighbour n of site s is higher than s  <=>  b(n) ^ b(s) = (i_s + j_s + par) & 1,
//   sigma_x(i,j) = +1 <=> b(i+1,j) ^ b(i,j) = (i+j+par) & 1, likewise sigma_y.
// A flip (h -> h +- 2) toggles b of that one site. One bit per site is the
// information content of the surface; the 2-bit slope format of the paper
// (Sec. 2.1) is kept as the exchange format of the C ABI.
//
// HBM layout of a lattice of lateral size L (bit-sliced cell rows):
//   storage cell = 4 x 4 sites; cell row R = sites with y in [4R, 4R+4), R < L/4;
//   block column K = 32 consecutive storage cells along x (128 sites), K < L/128;
//   plane p = (y%4) * 4 + x%4.
//   word(K, p, R) = lat[(K*16 + p) * (L/4) + R]; bit c of it is b of site
//   (128K + 4c + x%4, 4R + y%4).
// One word holds the bit of 32 cells, so one logic instruction updates 32
// cells ("multi-spin coding" of the bit-coded cellular automaton, Sec. 5).
// Lanes of a warp read consecutive R: a warp's load or store of one plane
// covers 128 contiguous bytes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kpz {

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplications whose high halves are mixed
// with the other two words and a round key advanced by two Weyl constants.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u, kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u, kPhiloxWeylB = 0xBB67AE85u;
constexpr int kPhiloxRounds = 10;

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < kPhiloxRounds; ++r) {
    const uint32_t hiA = __umulhi(kPhiloxMulA, c0), loA = kPhiloxMulA * c0;
    const uint32_t hiB = __umulhi(kPhiloxMulB, c2), loB = kPhiloxMulB * c2;
    const uint32_t n0 = hiB ^ c1 ^ k0;
    const uint32_t n2 = hiA ^ c3 ^ k1;
    c0 = n0; c1 = loB; c2 = n2; c3 = loA;
    k0 += kPhiloxWeylA; k1 += kPhiloxWeylB;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Philox4x32-10 with the ten round keys (k0 + r W_A, k1 + r W_B) read from
// shared memory as rk[r/2] = {key r, key r+1} (same output as philox()).
__device__ __forceinline__ uint4 philox_sk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint4* rk) {
#pragma unroll
  for (int r = 0; r < kPhiloxRounds; r += 2) {
    const uint4 k = rk[r >> 1];
    uint32_t hiA = __umulhi(kPhiloxMulA, c0), loA = kPhiloxMulA * c0;
    uint32_t hiB = __umulhi(kPhiloxMulB, c2), loB = kPhiloxMulB * c2;
    c0 = hiB ^ c1 ^ k.x; c1 = loB; c2 = hiA ^ c3 ^ k.y; c3 = loA;
    hiA = __umulhi(kPhiloxMulA, c0); loA = kPhiloxMulA * c0;
    hiB = __umulhi(kPhiloxMulB, c2); loB = kPhiloxMulB * c2;
    c0 = hiB ^ c1 ^ k.z; c1 = loB; c2 = hiA ^ c3 ^ k.w; c3 = loA;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Stream tags of the Philox counter word 0 (tag << 28 | index).
enum : uint32_t { kTagOrigin = 0u, kTagSet = 1u, kTagPos = 2u, kTagAcc = 3u, kTagPhase = 5u,
                  kTagClass = 6u, kTagClassAcc = 7u, kTagDeep = 8u };

constexpr uint32_t kTile = 128;      // tile edge in sites (device layer)
constexpr uint32_t kRounds = 16;     // single-hit rounds per sweep = sites per cell
constexpr uint32_t kPlanes = 16;     // bit planes per cell row

struct Geometry {
  uint32_t L;        // lateral size (power of two, >= 128)
  uint32_t NR;       // L/4 cell rows
  uint32_t NB;       // L/128 block columns
  uint32_t par;      // parity of h(0,0) of the start surface
  __host__ __device__ size_t word(uint32_t K, uint32_t p, uint32_t R) const {
    return ((size_t)K * kPlanes + p) * NR + R;
  }
};

__host__ __device__ constexpr uint32_t plane(uint32_t y4, uint32_t x4) { return y4 * 4u + x4; }

}  // namespace kpz
