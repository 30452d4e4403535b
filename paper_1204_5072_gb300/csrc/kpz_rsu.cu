// kpz_rsu.cu -- random-sequential updates on the GPU, equal bit for bit to
// making the attempts one at a time: the undecomposed dynamics that the
// decompositions of Sec. 3 (arXiv:1204.5072) approximate.
//
// Sweep s is the L^2 attempts a = 0 .. L^2 - 1 in order; attempt a draws
//   w = philox(4<<28, a, s, sample): site (w0 & (L-1), w1 & (L-1)), U = w2 >> 16
// and applies eq. (rule) there, a minimum rising when U < Tp and a maximum
// falling when U < Tq (the stream of the oracle's orc_rsu_run). An update at
// a site reads that site and its four neighbours and changes only the site,
// so attempt a depends on an earlier attempt b only when their sites are the
// same or neighbours. The sweep therefore runs in rounds: the attempts are
// bucketed by site (count, prefix sum, scatter, each site's list sorted), and
// in each round every site whose next attempt comes before the next attempt
// of each of its four neighbours makes it. Two such sites are never
// neighbours, and every attempt waits for all earlier attempts that touch
// it, so the lattice after the sweep is the one the sequential order gives
// (a conservative parallel discrete-event schedule). A round reads the
// per-site progress of the previous round (two buffers), so no site sees a
// neighbour's move of the same round. The host polls the number of attempts
// made after every few rounds; there is always progress (the earliest
// pending attempt of the sweep is always ready).
#include "kpz_rsu.h"

namespace kpz {
namespace {

constexpr uint32_t kTagRsu = 4u;
constexpr uint32_t kScanItems = 8, kScanThreads = 256, kScanBlock = kScanItems * kScanThreads;

__device__ __forceinline__ size_t site_word(const Geometry& g, uint32_t x, uint32_t y) {
  return g.word(x >> 7, plane(y & 3u, x & 3u), y >> 2);
}
__device__ __forceinline__ uint32_t bit_of(const uint32_t* lat, const Geometry& g, uint32_t x, uint32_t y) {
  return (__ldcg(lat + site_word(g, x, y)) >> ((x >> 2) & 31u)) & 1u;
}
__device__ __forceinline__ uint32_t sweep_index(const SweepParams& P) { return (uint32_t)(*P.t_dev) + P.s_add; }

// Site (row-major index y L + x) of attempt a.
__device__ __forceinline__ uint32_t attempt_site(const SweepParams& P, uint32_t s, uint32_t a, uint32_t& U) {
  const uint4 w = philox(kTagRsu << 28, a, s, P.sample, P.k0, P.k1);
  const uint32_t m = P.g.L - 1u;
  U = w.z >> 16;
  return (w.y & m) * P.g.L + (w.x & m);
}

__global__ void count_kernel(const SweepParams P, uint32_t n, uint32_t* cnt) {
  const uint32_t s = sweep_index(P);
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    uint32_t U;
    atomicAdd(cnt + attempt_site(P, s, a, U), 1u);
  }
}

// Exclusive prefix sum of cnt into off, in blocks of kScanBlock entries;
// bsum[b] receives block b's total.
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(const uint32_t* cnt, uint32_t n, uint32_t* off,
                                                                   uint32_t* bsum) {
  __shared__ uint32_t part[kScanThreads];
  const uint32_t base = blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], t = 0;
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? cnt[base + k] : 0u;
    t += v[k];
  }
  part[threadIdx.x] = t;
  __syncthreads();
  for (uint32_t d = 1; d < kScanThreads; d <<= 1) {
    const uint32_t x = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - t;
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    if (base + k < n) off[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1u) bsum[blockIdx.x] = part[threadIdx.x];
}

// Exclusive prefix sum of the block totals in place (one block of 1024 threads).
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t* bsum, uint32_t nb) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (nb + 1023u) / 1024u, b0 = threadIdx.x * per;
  uint32_t t = 0;
  for (uint32_t k = 0; k < per; ++k) t += b0 + k < nb ? bsum[b0 + k] : 0u;
  part[threadIdx.x] = t;
  __syncthreads();
  for (uint32_t d = 1; d < 1024u; d <<= 1) {
    const uint32_t x = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - t;
  for (uint32_t k = 0; k < per; ++k)
    if (b0 + k < nb) {
      const uint32_t v = bsum[b0 + k];
      bsum[b0 + k] = run;
      run += v;
    }
}

__global__ void scan_add_kernel(uint32_t* off, uint32_t n, const uint32_t* bsum) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    off[i] += bsum[i / kScanBlock];
}

// Attempt indices into their site's bucket (fill: zeroed per-site cursors).
__global__ void scatter_kernel(const SweepParams P, uint32_t n, const uint32_t* off, uint32_t* fill,
                               uint32_t* lst) {
  const uint32_t s = sweep_index(P);
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    uint32_t U;
    const uint32_t i = attempt_site(P, s, a, U);
    lst[off[i] + atomicAdd(fill + i, 1u)] = a;
  }
}

// Each site's bucket in increasing attempt order (insertion sort: a site has
// one attempt per sweep on average).
__global__ void sort_kernel(uint32_t n, const uint32_t* cnt, const uint32_t* off, uint32_t* lst) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t* b = lst + off[i];
    const uint32_t c = cnt[i];
    for (uint32_t k = 1; k < c; ++k) {
      const uint32_t v = b[k];
      uint32_t j = k;
      while (j > 0 && b[j - 1] > v) {
        b[j] = b[j - 1];
        --j;
      }
      b[j] = v;
    }
  }
}

// Next pending attempt of site i after `done` of its attempts, or UINT32_MAX.
__device__ __forceinline__ uint32_t next_attempt(const uint32_t* cnt, const uint32_t* off, const uint32_t* lst,
                                                 const uint32_t* done, uint32_t i) {
  const uint32_t d = done[i];
  return d < cnt[i] ? lst[off[i] + d] : 0xffffffffu;
}

// One round: every site whose next attempt is earlier than each neighbour's
// makes it. done_in / done_out: attempts made per site before / after.
__global__ void round_kernel(const SweepParams P, const uint32_t* cnt, const uint32_t* off, const uint32_t* lst,
                             const uint32_t* done_in, uint32_t* done_out, unsigned long long* made) {
  const uint32_t L = P.g.L, m = L - 1u, n = L * L, s = sweep_index(P);
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    bool fire = false;
    if (i < n) {
      const uint32_t d = done_in[i];
      const uint32_t a = d < cnt[i] ? lst[off[i] + d] : 0xffffffffu;
      const uint32_t x = i & m, y = i / L;
      if (a != 0xffffffffu) {
        fire = a < next_attempt(cnt, off, lst, done_in, y * L + ((x + m) & m)) &&
               a < next_attempt(cnt, off, lst, done_in, y * L + ((x + 1u) & m)) &&
               a < next_attempt(cnt, off, lst, done_in, ((y + m) & m) * L + x) &&
               a < next_attempt(cnt, off, lst, done_in, ((y + 1u) & m) * L + x);
      }
      if (fire) {
        uint32_t U;
        attempt_site(P, s, a, U);
        // Eq. (rule) on the height bits: neighbour n is higher iff b(n) ^ b(s) == parity(s).
        const uint32_t bs = bit_of(P.lat, P.g, x, y), hp = (x + y + P.g.par) & 1u;
        const bool hl = (bit_of(P.lat, P.g, (x + m) & m, y) ^ bs) == hp;
        const bool hr = (bit_of(P.lat, P.g, (x + 1u) & m, y) ^ bs) == hp;
        const bool hd = (bit_of(P.lat, P.g, x, (y + m) & m) ^ bs) == hp;
        const bool hu = (bit_of(P.lat, P.g, x, (y + 1u) & m) ^ bs) == hp;
        const bool is_min = hl && hr && hd && hu, is_max = !hl && !hr && !hd && !hu;
        if ((is_min && U < P.Tp) || (is_max && U < P.Tq)) {
          atomicXor(P.lat + site_word(P.g, x, y), 1u << ((x >> 2) & 31u));
          if (i == 0u) atomicAdd(P.h00, (unsigned long long)(long long)(is_min ? 2 : -2));
        }
      }
      done_out[i] = done_in[i] + (fire ? 1u : 0u);
    }
    const uint32_t warp_made = __popc(__ballot_sync(0xffffffffu, fire));
    if ((threadIdx.x & 31u) == 0u && warp_made) atomicAdd(made, (unsigned long long)warp_made);
  }
}

unsigned grid_for(uint32_t n, unsigned block) {
  const uint64_t b = ((uint64_t)n + block - 1) / block;
  return (unsigned)(b > 152u * 32u ? 152u * 32u : (b ? b : 1));
}

}  // namespace

size_t rsu_scratch_bytes(uint32_t L) {
  const size_t n = (size_t)L * L;
  return (5 * n + (n + kScanBlock - 1) / kScanBlock + 4) * sizeof(uint32_t) + 64;
}

cudaError_t launch_sweep_rsu(const SweepParams& P, void* scratch, cudaStream_t st) {
  const uint32_t L = P.g.L, n = L * L;
  uint32_t* cnt = static_cast<uint32_t*>(scratch);
  uint32_t* off = cnt + n;
  uint32_t* lst = off + n;
  uint32_t* da = lst + n;
  uint32_t* db = da + n;
  uint32_t* bsum = db + n;
  const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
  unsigned long long* made = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(bsum + nb) + 15u) & ~uintptr_t(15));
  cudaError_t e;
  if ((e = cudaMemsetAsync(cnt, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(da, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(made, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  count_kernel<<<grid_for(n, 256), 256, 0, st>>>(P, n, cnt);
  scan_blocks_kernel<<<nb, kScanThreads, 0, st>>>(cnt, n, off, bsum);
  scan_sums_kernel<<<1, 1024, 0, st>>>(bsum, nb);
  scan_add_kernel<<<grid_for(n, 256), 256, 0, st>>>(off, n, bsum);
  scatter_kernel<<<grid_for(n, 256), 256, 0, st>>>(P, n, off, da, lst);
  sort_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, cnt, off, lst);
  if ((e = cudaMemsetAsync(da, 0, n * sizeof(uint32_t), st)) != cudaSuccess) return e;
  count_launch(6);
  // Rounds, polled every kPoll: the sweep is done when all n attempts are made.
  constexpr int kPoll = 8;
  unsigned long long h_made = 0;
  uint32_t* cur = da;
  uint32_t* nxt = db;
  for (uint64_t rounds = 0; h_made < n; rounds += kPoll) {
    // A round always progresses and a sweep needs a few dozen; the bound only
    // turns a defect into an error instead of an endless loop.
    if (rounds >= (1u << 16)) return cudaErrorUnknown;
    for (int k = 0; k < kPoll; ++k) {
      round_kernel<<<grid_for(n, 256), 256, 0, st>>>(P, cnt, off, lst, cur, nxt, made);
      uint32_t* t = cur;
      cur = nxt;
      nxt = t;
    }
    count_launch(kPoll);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&h_made, made, sizeof(h_made), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace kpz
