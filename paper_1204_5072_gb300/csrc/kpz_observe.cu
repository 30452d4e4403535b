// kpz_observe.cu -- flat start, packed import/export, heights and exact W^2.
//
// Sec. 2.1 of arXiv:1204.5072: flat start with periodic boundaries, heights
// reconstructed from the slopes, squared interface width eq. (Wdef).
// Heights are built in the gauge h(0,0) = 0: first down column 0,
//   h(0,j) = sum_{k<j} sigma_y(0,k),
// then along each row, h(i,j) = h(0,j) + sum_{l<i} sigma_x(l,j); on a valid
// (curl-free) surface this equals any other path sum.
#include "kpz_internal.h"

namespace kpz {
namespace {

// Flat start: h = (i+j) & 1, so every slope is +1 where i+j is even. In the
// bit-sliced layout the parity of a site is (x%4 + y%4) % 2, the same for all
// 32 cells of a word.
__global__ void init_flat_kernel(uint4* lat4, Geometry g, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t w = i * 4;                 // 4 consecutive words share K and p
    const uint32_t p = (uint32_t)((w / g.NR) & 31u);
    const uint32_t y4 = p >> 3, x4 = (p >> 1) & 3u;
    const uint32_t v = ((x4 + y4) & 1u) ? 0u : ~0u;
    lat4[i] = make_uint4(v, v, v, v);
  }
}

// One packed word (16 sites of row j) per thread.
__global__ void export_kernel(const uint32_t* __restrict__ lat, Geometry g, uint32_t j0,
                              uint32_t nrows, uint32_t* __restrict__ packed) {
  const uint32_t wpr = g.L / 16;
  const size_t n = (size_t)nrows * wpr;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const uint32_t j = j0 + (uint32_t)(idx / wpr), wi = (uint32_t)(idx % wpr);
    const uint32_t K = wi >> 3, c0 = (wi & 7u) * 4u, R = j >> 2, y4 = j & 3u;
    uint32_t out = 0;
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4)
#pragma unroll
      for (uint32_t sg = 0; sg < 2; ++sg) {
        const uint32_t P = lat[g.word(K, plane(y4, x4, sg), R)] >> c0;
#pragma unroll
        for (uint32_t jc = 0; jc < 4; ++jc)
          out |= ((P >> jc) & 1u) << (2u * (4u * jc + x4) + sg);
      }
    packed[idx] = out;
  }
}

// One lattice word (K, p, R) per thread for cell rows [R0, R0 + nR), gathered
// from 8 packed words of the band that starts at row 4*R0.
__global__ void import_kernel(uint32_t* __restrict__ lat, Geometry g, uint32_t R0, uint32_t nR,
                              const uint32_t* __restrict__ packed) {
  const size_t n = (size_t)nR * 32u * g.NB;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const uint32_t R = R0 + (uint32_t)(idx % nR);
    const size_t rest = idx / nR;
    const uint32_t p = (uint32_t)(rest & 31u), K = (uint32_t)(rest >> 5);
    const size_t w = g.word(K, p, R);
    const uint32_t y4 = p >> 3, x4 = (p >> 1) & 3u, sg = p & 1u;
    const uint32_t j = 4u * (R - R0) + y4;
    const uint32_t* row = packed + (size_t)j * (g.L / 16) + 8u * K;
    uint32_t v = 0;
#pragma unroll
    for (uint32_t q = 0; q < 8; ++q) {
      const uint32_t pw = row[q];
#pragma unroll
      for (uint32_t jc = 0; jc < 4; ++jc)
        v |= ((pw >> (2u * (4u * jc + x4) + sg)) & 1u) << (4u * q + jc);
    }
    lat[w] = v;
  }
}

// h(0,j) for all rows j: one block, chunked sequential sums + block scan.
__global__ void col0_kernel(const uint32_t* __restrict__ lat, Geometry g, int32_t* __restrict__ col0) {
  __shared__ int32_t part[1024];
  const uint32_t nt = blockDim.x, t = threadIdx.x;
  const uint32_t chunk = (g.L + nt - 1) / nt;
  const uint32_t j0 = t * chunk, j1 = min(g.L, j0 + chunk);
  int32_t sum = 0;
  for (uint32_t j = j0; j < j1; ++j) {
    const uint32_t bit = lat[g.word(0, plane(j & 3u, 0, 1), j >> 2)] & 1u;  // sigma_y(0,j)
    sum += 2 * (int32_t)bit - 1;
  }
  part[t] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < nt; off <<= 1) {   // inclusive Hillis-Steele scan
    const int32_t v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t h = (t == 0) ? 0 : part[t - 1];
  for (uint32_t j = j0; j < j1; ++j) {
    col0[j] = h;
    const uint32_t bit = lat[g.word(0, plane(j & 3u, 0, 1), j >> 2)] & 1u;
    h += 2 * (int32_t)bit - 1;
  }
}

// Exact S1 = sum h and S2 = sum h^2 (eq. Wdef). Lane <-> row j = 4R + y4 with
// consecutive R per warp (coalesced plane loads); each 128-site block is
// summed relative to its first site in 32-bit, then promoted to 64-bit.
__global__ void roughness_kernel(const uint32_t* __restrict__ lat, Geometry g,
                                 const int32_t* __restrict__ col0,
                                 unsigned long long* __restrict__ acc) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t y4 = gw & 3u, R = (gw >> 2) * 32u + lane;
  long long s1 = 0;
  unsigned long long s2 = 0;
  if (R < g.NR) {
    const uint32_t j = 4u * R + y4;
    long long H = col0[j];
    for (uint32_t K = 0; K < g.NB; ++K) {
      uint32_t P[4];
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) P[x4] = __ldcg(lat + g.word(K, plane(y4, x4, 0), R));
      int32_t h = 0, a1 = 0, a2 = 0;
#pragma unroll 8
      for (uint32_t c = 0; c < 32; ++c)
#pragma unroll
        for (uint32_t x4 = 0; x4 < 4; ++x4) {
          a1 += h;
          a2 += h * h;
          h += 2 * (int32_t)((P[x4] >> c) & 1u) - 1;
        }
      s1 += 128 * H + a1;
      s2 += (unsigned long long)(128 * H * H + 2 * H * (long long)a1 + (long long)a2);
      H += h;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (lane == 0 && (s1 != 0 || s2 != 0)) {
    atomicAdd(&acc[0], (unsigned long long)s1);
    const unsigned long long old = atomicAdd(&acc[1], s2);
    if (old + s2 < old) atomicAdd(&acc[2], 1ull);
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
    for (uint32_t x4 = 0; x4 < 4; ++x4) P[x4] = lat[g.word(K, plane(y4, x4, 0), R)];
    for (uint32_t c = 0; c < 32; ++c)
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) {
        o[128u * K + 4u * c + x4] = h;
        h += 2 * (int64_t)((P[x4] >> c) & 1u) - 1;
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
  const size_t n4 = (size_t)g.L * g.L / 64;
  init_flat_kernel<<<grid_for(n4, 256), 256, 0, st>>>(reinterpret_cast<uint4*>(lat), g, n4);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_export_packed(const uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 uint32_t* packed, cudaStream_t st) {
  export_kernel<<<grid_for((size_t)nrows * (g.L / 16), 256), 256, 0, st>>>(lat, g, j0, nrows, packed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_import_packed(uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 const uint32_t* packed, cudaStream_t st) {
  const uint32_t R0 = j0 / 4u, nR = nrows / 4u;
  import_kernel<<<grid_for((size_t)nR * 32u * g.NB, 256), 256, 0, st>>>(lat, g, R0, nR, packed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_col0(const uint32_t* lat, Geometry g, int32_t* col0, cudaStream_t st) {
  col0_kernel<<<1, 1024, 0, st>>>(lat, g, col0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_roughness(const uint32_t* lat, Geometry g, int32_t* col0,
                             unsigned long long* acc, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  col0_kernel<<<1, 1024, 0, st>>>(lat, g, col0);
  count_launch();
  const uint32_t warps = 4u * ((g.NR + 31u) / 32u);
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
