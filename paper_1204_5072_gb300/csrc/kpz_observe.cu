// kpz_observe.cu -- flat start, packed import/export, heights and exact W^2.
//
// Sec. 2.1 of arXiv:1204.5072: flat start with periodic boundaries, heights
// reconstructed from the slopes, squared interface width eq. (Wdef).
// The lattice holds one bit per site, b = (h >> 1) & 1 (kpz_common.cuh); the
// slopes follow from neighbouring bits and the site parity (i + j + par) & 1.
// Heights are built in the gauge h(0,0) = 0: first down column 0,
//   h(0,j) = sum_{k<j} sigma_y(0,k),
// then along each row, h(i,j) = h(0,j) + sum_{l<i} sigma_x(l,j); on a valid
// (curl-free) surface this equals any other path sum.
#include <algorithm>

#include "kpz_internal.h"
#include "kpz_w2.cuh"

namespace kpz {
namespace {

// Bit b of site (i, j) (i < L, j < L).
__device__ __forceinline__ uint32_t site_bit(const uint32_t* lat, const Geometry& g, uint32_t i,
                                             uint32_t j) {
  return (lat[g.word(i >> 7, plane(j & 3u, i & 3u), j >> 2)] >> ((i >> 2) & 31u)) & 1u;
}

// Flat start h = (i+j) & 1: h >> 1 = 0 everywhere.
__global__ void init_flat_kernel(uint4* lat4, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x)
    lat4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Bits of 4 consecutive cells (starting at cell c0) of a plane, spread to
// positions 4*jc (jc = cell offset): the row-major order of sites 4jc + x4.
__device__ __forceinline__ uint32_t spread4(uint32_t n) {
  return (n & 1u) | ((n & 2u) << 3) | ((n & 4u) << 6) | ((n & 8u) << 9);
}

// Interleave: bit k of a -> bit 2k, for a < 2^16.
__device__ __forceinline__ uint32_t part1by1(uint32_t a) {
  a = (a | (a << 8)) & 0x00FF00FFu;
  a = (a | (a << 4)) & 0x0F0F0F0Fu;
  a = (a | (a << 2)) & 0x33333333u;
  a = (a | (a << 1)) & 0x55555555u;
  return a;
}

// Block columns of one import/export block: warp w of a block takes block
// columns [w KS, (w + 1) KS), KS = NB / min(kIoSegs, NB).
constexpr uint32_t kIoSegs = 16;

// Rows j = 4R + y4 of a band for 32 consecutive cell rows R (lane = R - R0)
// and one y4 (blockIdx.x = 4 group + y4): a warp's loads of one plane word are
// 128 contiguous bytes, and each lane writes its row's 8 packed words of a
// block column (32 contiguous bytes).
__global__ void __launch_bounds__(32 * kIoSegs) export_kernel(const uint32_t* __restrict__ lat, Geometry g,
                                                              uint32_t j0, uint32_t nrows,
                                                              uint32_t* __restrict__ packed) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t S = min(kIoSegs, g.NB), KS = g.NB / S;
  const uint32_t y4 = blockIdx.x & 3u, rr = 32u * (blockIdx.x >> 2) + lane;
  if (w >= S || 4u * rr >= nrows) return;
  const uint32_t R = j0 / 4u + rr, j = 4u * R + y4;
  const uint32_t y4n = (y4 + 1u) & 3u, Rn = (y4 == 3u) ? ((R + 1u) & (g.NR - 1u)) : R;   // row j + 1
  // parity of site 16 wi + k is (k + j + par) & 1; a neighbour is higher iff
  // the bits differ by that parity, so sigma = +1 <=> b(next) ^ b ^ parity == 0
  const uint32_t odd = ((j + g.par) & 1u) ? 0x5555u : 0xAAAAu;
  uint4* out = reinterpret_cast<uint4*>(packed + (size_t)(4u * rr + y4) * (g.L / 16u));
  for (uint32_t K = w * KS; K < (w + 1u) * KS; ++K) {
    uint32_t A[4], B[4];
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4) {
      A[x4] = lat[g.word(K, plane(y4, x4), R)];
      B[x4] = lat[g.word(K, plane(y4n, x4), Rn)];
    }
    const uint32_t nxt = lat[g.word((K + 1u) & (g.NB - 1u), plane(y4, 0), R)] & 1u;   // site 128(K+1)
    uint32_t o[8];
#pragma unroll
    for (uint32_t q = 0; q < 8; ++q) {   // packed word q: sites 16q + k = cells 4q + k/4, x4 = k%4
      uint32_t r0 = 0, r1 = 0;
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) {
        r0 |= spread4((A[x4] >> (4u * q)) & 0xFu) << x4;
        r1 |= spread4((B[x4] >> (4u * q)) & 0xFu) << x4;
      }
      r0 |= (q < 7u ? (A[0] >> (4u * q + 4u)) & 1u : nxt) << 16;
      const uint32_t sx = ~((r0 >> 1) ^ r0 ^ odd) & 0xFFFFu;
      const uint32_t sy = ~(r1 ^ r0 ^ odd) & 0xFFFFu;
      o[q] = part1by1(sx) | (part1by1(sy) << 1);
    }
    out[2u * K] = make_uint4(o[0], o[1], o[2], o[3]);
    out[2u * K + 1u] = make_uint4(o[4], o[5], o[6], o[7]);
  }
}

// Absolute heights modulo 4 down column 0 for rows [j0, j0 + nrows) of a
// packed band; hcar holds h(0, j0) mod 4 on entry and h(0, j0 + nrows) mod 4
// on exit. One block.
__global__ void import_col_kernel(const uint32_t* __restrict__ packed, Geometry g, uint32_t nrows,
                                  uint32_t* __restrict__ hcar, int32_t* __restrict__ hcol) {
  __shared__ int32_t part[1024];
  const uint32_t nt = blockDim.x, t = threadIdx.x, wpr = g.L / 16;
  const uint32_t chunk = (nrows + nt - 1) / nt;
  const uint32_t r0 = min(nrows, t * chunk), r1 = min(nrows, r0 + chunk);
  int32_t sum = 0;
  for (uint32_t r = r0; r < r1; ++r) sum += ((packed[(size_t)r * wpr] >> 1) & 1u) ? 1 : -1;
  part[t] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < nt; off <<= 1) {
    const int32_t v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  const int32_t base = (int32_t)*hcar;
  int32_t h = base + ((t == 0) ? 0 : part[t - 1]);
  for (uint32_t r = r0; r < r1; ++r) {
    hcol[r] = h & 3;
    h += ((packed[(size_t)r * wpr] >> 1) & 1u) ? 1 : -1;
  }
  __syncthreads();
  if (t == nt - 1) *hcar = (uint32_t)((base + part[nt - 1]) & 3);
}

// The 16 x-slopes of a packed word (its even bits) at bits 0..15.
__device__ __forceinline__ uint32_t even_bits(uint32_t a) {
  a &= 0x55555555u;
  a = (a | (a >> 1)) & 0x33333333u;
  a = (a | (a >> 2)) & 0x0F0F0F0Fu;
  a = (a | (a >> 4)) & 0x00FF00FFu;
  return (a | (a >> 8)) & 0x0000FFFFu;
}

// Bits 0, 4, 8, 12 of v at bits 0..3.
__device__ __forceinline__ uint32_t gather4(uint32_t v) {
  v &= 0x1111u;
  v = (v | (v >> 3)) & 0x0303u;
  return (v | (v >> 6)) & 0xFu;
}

// Bits of the rows of a packed band, laid out as in export_kernel. Along row
// j, h(i,j) = h(0,j) - i + 2 U(i,j) with U(i,j) the number of +1 x-slopes
// left of i, so b(i,j) = bit 1 of (h(0,j) - i) mod 4, XOR U(i,j) mod 2: a
// prefix XOR of the x-slope bits. Each warp first takes the parity of its
// block columns' x-slopes; the parities of the segments before it give its
// carry.
__global__ void __launch_bounds__(32 * kIoSegs) import_rows_kernel(uint32_t* __restrict__ lat, Geometry g,
                                                                   uint32_t j0, uint32_t nrows,
                                                                   const uint32_t* __restrict__ packed,
                                                                   const int32_t* __restrict__ hcol) {
  __shared__ uint32_t seg_par[kIoSegs][32];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t S = min(kIoSegs, g.NB), KS = g.NB / S;
  const uint32_t y4 = blockIdx.x & 3u, rr = 32u * (blockIdx.x >> 2) + lane;
  const bool live = w < S && 4u * rr < nrows;
  const uint32_t r = 4u * rr + y4;   // row within the band
  const uint4* row = reinterpret_cast<const uint4*>(packed + (size_t)(live ? r : 0u) * (g.L / 16u));
  uint32_t x = 0;
  if (live)
    for (uint32_t K = w * KS; K < (w + 1u) * KS; ++K) {
      const uint4 a = row[2u * K], b = row[2u * K + 1u];
      x ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
    }
  seg_par[w][lane] = __popc(x & 0x55555555u) & 1u;
  __syncthreads();
  if (!live) return;
  uint32_t carry = 0;   // parity of the +1 x-slopes left of the segment
  for (uint32_t v = 0; v < w; ++v) carry ^= seg_par[v][lane];
  // bit 1 of (h(0,j) - k) mod 4 for k = 0..15 (period 4; 16 wi = 0 mod 4)
  const uint32_t pat = ((0x39C6u >> (4u * ((uint32_t)hcol[r] & 3u))) & 0xFu) * 0x1111u;
  const uint32_t R = j0 / 4u + rr;
  for (uint32_t K = w * KS; K < (w + 1u) * KS; ++K) {
    const uint4 a = row[2u * K], b = row[2u * K + 1u];
    const uint32_t pw[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t W[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (uint32_t q = 0; q < 8; ++q) {   // sites 128K + 16q + k = cell 4q + k/4, x4 = k%4
      uint32_t e = even_bits(pw[q]);
      e ^= e << 1;
      e ^= e << 2;
      e ^= e << 4;
      e ^= e << 8;                       // bit k: parity of the x-slopes 0..k of the word
      const uint32_t bits = (((e << 1) ^ (0u - carry)) & 0xFFFFu) ^ pat;
      carry ^= (e >> 15) & 1u;
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) W[x4] |= gather4(bits >> x4) << (4u * q);
    }
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4) lat[g.word(K, plane(y4, x4), R)] = W[x4];
  }
}

// h(0,j) for all rows j, gauge h(0,0) = 0: one block; thread t owns rows
// [t chunk, (t+1) chunk) in pieces of 32. A piece's 32 bits b(0, j) are loaded
// at once into a mask; its steps sigma_y(0, j) = +1 where b(0,j) ^ b(0,j+1)
// equals the parity of j + par, so the piece's height change is
// 2 popc(E) - 32; a block scan of the chunk sums gives each chunk's start.
constexpr uint32_t kCol0Threads = 1024;

__global__ void __launch_bounds__(kCol0Threads) col0_kernel(const uint32_t* __restrict__ lat, Geometry g,
                                                           int32_t* __restrict__ col0) {
  __shared__ int32_t part[kCol0Threads];
  const uint32_t nt = blockDim.x, t = threadIdx.x;
  const uint32_t chunk = g.L / nt;                 // multiple of 32
  const uint32_t j0 = t * chunk, pieces = chunk / 32u;
  const uint32_t parpat = ((g.par & 1u) ? 0x55555555u : 0xAAAAAAAAu);  // bit i: (j0+32p+i+par) odd
  auto piece_steps = [&](uint32_t jp) -> uint32_t {   // E bits of rows jp .. jp+31
    // Rows jp + 4r + y4 (r < 8): words R0 + r of plane (y4, 0), R0 = jp/4 a
    // multiple of 8, read as two 16-byte vectors per plane.
    uint32_t b = 0;
#pragma unroll
    for (uint32_t y4 = 0; y4 < 4u; ++y4) {
      const uint4* v = reinterpret_cast<const uint4*>(lat + g.word(0, plane(y4, 0), jp >> 2));
      const uint4 lo = __ldcg(v), hi = __ldcg(v + 1);
      const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (uint32_t r = 0; r < 8u; ++r) b |= (w[r] & 1u) << (4u * r + y4);
    }
    const uint32_t jn = (jp + 32u) & (g.L - 1u);
    const uint32_t bn = __ldcg(lat + g.word(0, plane(jn & 3u, 0), jn >> 2)) & 1u;
    return ~(b ^ ((b >> 1) | (bn << 31)) ^ parpat);
  };
  int32_t sum = 0;
  for (uint32_t p = 0; p < pieces; ++p) sum += 2 * __popc(piece_steps(j0 + 32u * p)) - 32;
  part[t] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < nt; off <<= 1) {   // inclusive Hillis-Steele scan
    const int32_t v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t h = (t == 0) ? 0 : part[t - 1];
  for (uint32_t p = 0; p < pieces; ++p) {
    const uint32_t E = piece_steps(j0 + 32u * p);
    int32_t* o = col0 + j0 + 32u * p;
#pragma unroll 8
    for (uint32_t i = 0; i < 32u; ++i) {
      o[i] = h;
      h += ((E >> i) & 1u) ? 1 : -1;
    }
  }
}

// Work split: warp -> (y4, 8 consecutive storage rows R); lane -> row R + (lane & 7)
// and segment q = lane >> 3 of kSegs block columns each; a segment's start
// height is col0 plus the height changes of the segments before it (a scan
// over the 4 lanes of the row).
constexpr uint32_t kRowsPerWarp = 8, kSegs = 4;

__global__ void __launch_bounds__(256) roughness_kernel(const uint32_t* __restrict__ lat, Geometry g,
                                                        const int32_t* __restrict__ col0,
                                                        unsigned long long* __restrict__ acc) {
  __shared__ uint32_t tab[w2::kRunTableWords];
  w2::fill_run_table(tab);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t* tl = tab + lane;
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t y4 = gw & 3u, R = (gw >> 2) * kRowsPerWarp + (lane & (kRowsPerWarp - 1u));
  const uint32_t q = lane / kRowsPerWarp;
  const uint32_t seg = (g.NB + kSegs - 1u) / kSegs;               // block columns per segment
  const uint32_t K0 = q * seg, K1 = min(g.NB, K0 + seg);
  const bool active = R < g.NR && K0 < K1;
  long long s1 = 0, s2 = 0, dH = 0;   // relative to the segment's first site
  if (active) {
    uint32_t P[4], Pn[4];
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4) {
      P[x4] = __ldcg(lat + g.word(K0, plane(y4, x4), R));
      Pn[x4] = __ldcg(lat + g.word((K0 + 1u) & (g.NB - 1u), plane(y4, x4), R));
    }
    const uint32_t j = 4u * R + y4;
    for (uint32_t K = K0; K < K1; ++K) {
      uint32_t Pnn[4];   // two blocks ahead
      const uint32_t K2 = (K + 2u) & (g.NB - 1u);
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) Pnn[x4] = __ldcg(lat + g.word(K2, plane(y4, x4), R));
      uint32_t S[4];
      w2::sigma_x_planes(P, Pn[0] & 1u, j, g.par, S);
      int32_t h, a1, a2;
      w2::block_sums(tl, S, h, a1, a2);
      s1 += 128 * dH + a1;
      s2 += 128 * dH * dH + 2 * dH * (long long)a1 + (long long)a2;
      dH += h;
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) { P[x4] = Pn[x4]; Pn[x4] = Pnn[x4]; }
    }
  }
  // Start height of this segment: col0[j] + height changes of the row's earlier segments.
  long long pre = dH;
#pragma unroll
  for (uint32_t d = kRowsPerWarp; d < 32u; d <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, pre, d);
    if (lane >= d) pre += v;
  }
  long long t1 = 0;
  unsigned long long t2 = 0;
  if (active) {
    const long long H0 = (long long)col0[4u * R + y4] + (pre - dH);
    const long long n = 128ll * (K1 - K0);
    t1 = n * H0 + s1;
    t2 = (unsigned long long)(n * H0 * H0 + 2 * H0 * s1 + s2);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, off);
    t2 += __shfl_xor_sync(0xffffffffu, t2, off);
  }
  if (lane == 0 && (t1 != 0 || t2 != 0)) {
    atomicAdd(&acc[0], (unsigned long long)t1);
    const unsigned long long old = atomicAdd(&acc[1], t2);
    if (old + t2 < old) atomicAdd(&acc[2], 1ull);
  }
}

__global__ void heights_kernel(const uint32_t* __restrict__ lat, Geometry g,
                               const int32_t* __restrict__ col0, uint32_t j0, uint32_t nrows,
                               const unsigned long long* __restrict__ h00, int64_t* __restrict__ out) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const uint32_t j = j0 + r, R = j >> 2, y4 = j & 3u;
  int64_t h = col0[j] + (h00 ? (int64_t)*h00 : 0);
  int64_t* o = out + (size_t)r * g.L;
  for (uint32_t K = 0; K < g.NB; ++K) {
    uint32_t P[4];
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4) P[x4] = lat[g.word(K, plane(y4, x4), R)];
    const uint32_t nxt = site_bit(lat, g, (128u * K + 128u) & (g.L - 1u), j);
    uint32_t S[4];
    w2::sigma_x_planes(P, nxt, j, g.par, S);
    for (uint32_t c = 0; c < 32; ++c)
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) {
        o[128u * K + 4u * c + x4] = h;
        h += 2 * (int64_t)((S[x4] >> c) & 1u) - 1;
      }
  }
}

unsigned grid_for(size_t n, unsigned block) {
  size_t b = (n + block - 1) / block;
  if (b > 152u * 64u) b = 152u * 64u;
  return (unsigned)(b ? b : 1);
}

}  // namespace

cudaError_t launch_init_flat(uint32_t* lat, Geometry g, cudaStream_t st) {
  const size_t n4 = (size_t)g.L * g.L / 128;   // L^2 bits = L^2/128 uint4
  init_flat_kernel<<<grid_for(n4, 256), 256, 0, st>>>(reinterpret_cast<uint4*>(lat), n4);
  count_launch();
  return cudaGetLastError();
}

// Both conversions take j0 and nrows as multiples of 4 (whole cell rows) and a
// 16-byte aligned packed band.
cudaError_t launch_export_packed(const uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 uint32_t* packed, cudaStream_t st) {
  export_kernel<<<4u * ((nrows / 4u + 31u) / 32u), 32u * kIoSegs, 0, st>>>(lat, g, j0, nrows, packed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_import_packed(uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 const uint32_t* packed, uint32_t* hcar, int32_t* hcol,
                                 cudaStream_t st) {
  import_col_kernel<<<1, 1024, 0, st>>>(packed, g, nrows, hcar, hcol);
  count_launch();
  import_rows_kernel<<<4u * ((nrows / 4u + 31u) / 32u), 32u * kIoSegs, 0, st>>>(lat, g, j0, nrows, packed, hcol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_col0(const uint32_t* lat, Geometry g, int32_t* col0, cudaStream_t st) {
  col0_kernel<<<1, std::min(kCol0Threads, g.L / 32u), 0, st>>>(lat, g, col0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_roughness(const uint32_t* lat, Geometry g, int32_t* col0,
                             unsigned long long* acc, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  col0_kernel<<<1, std::min(kCol0Threads, g.L / 32u), 0, st>>>(lat, g, col0);
  count_launch();
  const uint32_t warps = 4u * ((g.NR + kRowsPerWarp - 1u) / kRowsPerWarp);
  const uint32_t wpc = 8;
  roughness_kernel<<<(warps + wpc - 1) / wpc, wpc * 32, 0, st>>>(lat, g, col0, acc);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_heights(const uint32_t* lat, Geometry g, const int32_t* col0, uint32_t j0,
                           uint32_t nrows, const unsigned long long* h00, int64_t* out,
                           cudaStream_t st) {
  heights_kernel<<<(nrows + 127) / 128, 128, 0, st>>>(lat, g, col0, j0, nrows, h00, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace kpz
