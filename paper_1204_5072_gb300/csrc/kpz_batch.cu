// kpz_batch.cu -- many independent realisations in one persistent launch.
//
// Each realisation is its own L x L lattice with its own rates, key and run
// length (Sec. 2.1 model, Sec. 3 decomposition, exactly as kpz_run sweeps it).
// One cooperative launch keeps a fixed set of warps resident; they take work
// items from one global queue, in order:
//   phase g = 0, 1, ..., T_max:  [W^2 bands of every realisation that samples
//   at time g] [sweep g: every tile run of every realisation with T_r > g]
// A tile run of sweep g of realisation r waits until all tile runs of its
// sweep g-1 and all its W^2 bands up to time g are done (per-realisation
// counters); a W^2 band at time g waits for sweep g-1. Items only wait on
// items earlier in the queue, which resident warps already hold, so the wait
// always ends; it is still bounded in time and, if the bound is hit, every
// warp stops and the host gets KPZ_ETIMEOUT. Small lattices thus run beside
// large ones instead of leaving most of the GPU idle, and no launch per sweep
// is needed. The scheduling knobs (tiles per run, warps per block, blocks per
// SM) do not change any result.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "kpz.h"
#include "kpz_run.cuh"
#include "kpz_w2.cuh"

namespace kpz {
namespace batch {

struct Segment {                // consecutive phases with the same item layout
  unsigned long long base;      // queue index of the first item
  uint32_t g0, nph;             // phases g0 .. g0 + nph - 1
  uint32_t size;                // items per phase
  uint32_t has_sample;          // 1: phase g0 starts with W^2 bands (then nph = 1)
  uint32_t As, Aw;              // realisations (sorted prefix) sampling / sweeping here
  uint32_t nsamp;               // sample times <= g (sweeps of these phases need them done)
};

struct Real {                   // one realisation, sorted by run length, longest first
  SweepParams P;                // lattice, geometry, rates, key, tiles per run
  uint32_t n_items;             // tile runs per sweep
  uint32_t nb;                  // W^2 bands per sample (L/128 rows of 128)
  uint32_t general;             // rates other than p = 1, q = 0
};

struct Plan {
  const Segment* seg;
  uint32_t nseg;
  const Real* real;
  const unsigned long long* PW;  // prefix sums of n_items over sorted realisations
  const unsigned long long* PS;  // prefix sums of nb
  unsigned long long total;      // items in the queue
  unsigned long long* head;      // next queue index
  unsigned long long* sweep_done;
  unsigned long long* sample_done;
  unsigned long long* acc;       // [band of all realisations][sample index][D, S1, S2] (band-relative)
  uint32_t nG;                   // sample times
  int* err;                      // set to 1 when a wait ran out of time
  unsigned long long timeout_ns;
  int block;                     // test hook: realisation whose waits can never succeed
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lane 0: wait until *c >= target, at most Q.timeout_ns; false on timeout or
// when another warp has already reported one.
__device__ bool wait_ge(const unsigned long long* c, unsigned long long target, const Plan& Q) {
  if (ld_acquire(c) >= target) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    __nanosleep(200);
    if (ld_acquire(c) >= target) return true;
    if (*(volatile int*)Q.err) return false;
    if (now_ns() - t0 > Q.timeout_ns) {
      atomicExch(Q.err, 1);
      return false;
    }
  }
}

template <typename T>
__device__ __forceinline__ uint32_t upper_index(const T* a, uint32_t n, T v) {
  // largest i in [0, n) with a[i] <= v (a[0] <= v, ascending)
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// b(0, m): height bit of site (0, m).
__device__ __forceinline__ uint32_t col0_bit(const uint32_t* lat, const Geometry& g, uint32_t m) {
  return __ldcg(lat + g.word(0, plane(m & 3u, 0), m >> 2)) & 1u;
}
// sigma_y(0, m) as +-1 (Sec. 2.1 slopes from the height bits).
__device__ __forceinline__ int sigma_y0(const uint32_t* lat, const Geometry& g, uint32_t m) {
  const uint32_t b = col0_bit(lat, g, m), bn = col0_bit(lat, g, (m + 1u) & (g.L - 1u));
  return ((b ^ bn) == ((m + g.par) & 1u)) ? 1 : -1;
}

// W^2 band k of a lattice (rows 128k .. 128k+127; lane l takes cell row
// R = 32k + l, i.e. rows 4R .. 4R+3): the column-0 height change D over the
// band and the sums S1 = sum h, S2 = sum h^2 of its heights relative to
// h(0, 128k) (eq. Wdef). The host chains the bands: band k starts at the sum
// of the D of the bands above it. tl = the lane's copy of the run table.
__device__ void band_sums(const SweepParams& P, const uint32_t* tl, uint32_t k, uint32_t lane,
                          long long& d, long long& s1, unsigned long long& s2) {
  const Geometry g = P.g;
  const uint32_t* lat = P.lat;
  const uint32_t R = 32u * k + lane;
  int own[4], tot = 0;
#pragma unroll
  for (uint32_t y4 = 0; y4 < 4; ++y4) { own[y4] = sigma_y0(lat, g, 4u * R + y4); tot += own[y4]; }
  int incl = tot;  // inclusive scan over lanes
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if ((int)lane >= off) incl += v;
  }
  d = __shfl_sync(0xffffffffu, incl, 31);
  long long H0 = incl - tot;  // h(0, 4R) - h(0, 128k)
  s1 = 0;
  s2 = 0;
#pragma unroll 1
  for (uint32_t y4 = 0; y4 < 4; ++y4) {
    const uint32_t j = 4u * R + y4;
    long long H = H0;
    uint32_t Pl[4], Pn[4];
#pragma unroll
    for (uint32_t x4 = 0; x4 < 4; ++x4) {
      Pl[x4] = __ldcg(lat + g.word(0, plane(y4, x4), R));
      Pn[x4] = __ldcg(lat + g.word(1u & (g.NB - 1u), plane(y4, x4), R));
    }
    for (uint32_t K = 0; K < g.NB; ++K) {
      uint32_t Pnn[4];   // two blocks ahead
      const uint32_t K2 = (K + 2u) & (g.NB - 1u);
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) Pnn[x4] = __ldcg(lat + g.word(K2, plane(y4, x4), R));
      uint32_t S[4];  // bit c: sigma_x(128K + 4c + x4, j) = +1
      w2::sigma_x_planes(Pl, Pn[0] & 1u, j, g.par, S);
      int32_t h, a1, a2;
      w2::block_sums(tl, S, h, a1, a2);
      s1 += 128 * H + a1;
      s2 += (unsigned long long)(128 * H * H + 2 * H * (long long)a1 + (long long)a2);
      H += h;
#pragma unroll
      for (uint32_t x4 = 0; x4 < 4; ++x4) { Pl[x4] = Pn[x4]; Pn[x4] = Pnn[x4]; }
    }
    H0 += own[y4];
  }
}

// Per-warp shared memory. 16-byte aligned size: the slab copies are 16-byte
// cp.async writes, so every warp's slot must start on a 16-byte boundary.
template <int CR>
struct alignas(16) WarpSlot {
  run::WarpStage<CR> stage;
  SweepParams P;
  uint4 rk[kPhiloxRounds / 2];   // Philox round keys of the item's realisation
};
static_assert(sizeof(WarpSlot<1>) % 16 == 0 && sizeof(WarpSlot<2>) % 16 == 0,
              "warp slots must keep 16-byte alignment");

// CR = cell rows per lane: tiles of 128 x 128 CR sites.
template <int CR>
__global__ void __launch_bounds__(256, 2) batch_kernel(const __grid_constant__ Plan Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSlot<CR>& ws = reinterpret_cast<WarpSlot<CR>*>(smem_raw)[threadIdx.x >> 5];
  __shared__ uint32_t tab[w2::kRunTableWords];   // W^2 run table (kpz_w2.cuh)
  w2::fill_run_table(tab);
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = (*(volatile int*)Q.err) ? Q.total : atomicAdd(Q.head, 1ull);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= Q.total) break;

    // Decode the queue index: segment, phase g, sample band or tile run.
    uint32_t lo = 0, hi = Q.nseg;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (Q.seg[mid].base <= idx) lo = mid; else hi = mid;
    }
    const Segment sg = Q.seg[lo];
    const unsigned long long off = idx - sg.base;
    const uint32_t g = sg.g0 + (uint32_t)(off / sg.size);
    unsigned long long o = off % sg.size;
    const unsigned long long nsample = sg.has_sample ? Q.PS[sg.As] : 0ull;
    const bool is_sample = o < nsample;
    uint32_t i;
    unsigned long long k;
    if (is_sample) {
      i = upper_index(Q.PS, sg.As + 1u, o);
      k = o - Q.PS[i];
    } else {
      o -= nsample;
      i = upper_index(Q.PW, sg.Aw + 1u, o);
      k = o - Q.PW[i];
    }
    const Real* re = &Q.real[i];

    // Dependencies (lane 0 waits, the warp follows).
    int ok = 1;
    if (lane == 0) {
      unsigned long long need = (unsigned long long)g * re->n_items;
      if ((int)i == Q.block) need += 1ull;
      ok = wait_ge(&Q.sweep_done[i], need, Q);
      if (ok && !is_sample) ok = wait_ge(&Q.sample_done[i], (unsigned long long)sg.nsamp * re->nb, Q);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) break;
    // This realisation's parameters, read in place by the tile code.
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&re->P);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&ws.P);
      for (uint32_t w = lane; w < sizeof(SweepParams) / 4; w += 32u) dst[w] = src[w];
    }
    const uint32_t general = re->general;
    __syncwarp();
    // Its Philox round keys, read by the tile code from shared memory.
    if (lane < kPhiloxRounds / 2) {
      const uint32_t r2 = 2u * lane;
      ws.rk[lane] = make_uint4(ws.P.k0 + r2 * kPhiloxWeylA, ws.P.k1 + r2 * kPhiloxWeylB,
                               ws.P.k0 + (r2 + 1u) * kPhiloxWeylA, ws.P.k1 + (r2 + 1u) * kPhiloxWeylB);
    }
    __syncwarp();

    if (is_sample) {
      long long d, s1;
      unsigned long long s2;
      band_sums(ws.P, tab + lane, (uint32_t)k, lane, d, s1, s2);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0) {
        unsigned long long* a = Q.acc + ((size_t)(Q.PS[i] + k) * Q.nG + (sg.nsamp - 1u)) * 3u;
        a[0] = (unsigned long long)d;
        a[1] = (unsigned long long)s1;
        a[2] = s2;
      }
    } else {
      const uint32_t ty = (uint32_t)(k / ws.P.runs_x);
      const uint32_t tx0 = (uint32_t)(k - (unsigned long long)ty * ws.P.runs_x) * ws.P.run;
      // Device layer: this sweep's random tile origin (Sec. 3).
      const uint4 o = philox(kTagOrigin << 28, 0u, g, ws.P.sample, ws.P.k0, ws.P.k1);
      const uint32_t L = ws.P.g.L, ox = o.x & (L - 1u), oy = o.y & (L - 1u);
      if (general) run::sweep_run<true, CR, true, true>(ws.P, ws.stage, ws.rk, lane, g, ox, oy, ty, tx0, ws.P.run);
      else         run::sweep_run<false, CR, true, true>(ws.P, ws.stage, ws.rk, lane, g, ox, oy, ty, tx0, ws.P.run);
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(is_sample ? &Q.sample_done[i] : &Q.sweep_done[i], 1ull);
  }
}

}  // namespace batch
}  // namespace kpz

// --------------------------------------------------------------------------
// Host side.
// --------------------------------------------------------------------------
using namespace kpz;
using namespace kpz::batch;

struct kpz_batch {
  std::vector<kpz_spec> spec;        // caller order
  std::vector<uint32_t> order;       // sorted position -> caller index
  std::vector<uint64_t> times;       // sample times
  cudaStream_t stream = nullptr;
  int device = 0;
  uint32_t sms = 0;
  // knobs (execution only)
  uint32_t run_max = 4, wpc = 8, ctas_per_sm = 0, grid = 0;
  uint32_t cr = 1;                   // cell rows per lane: tiles of 128 x 128 cr
  uint64_t timeout_ns = 10ull * 1000000000ull;
  int block = -1;
  // device memory
  void* pool = nullptr;
  size_t pool_bytes = 0;
  size_t lat_bytes = 0;              // lattices at the start of the pool
  size_t bands = 0;                  // W^2 bands of all realisations (sum of L/128)
  Plan plan{};
  std::vector<Real> real;            // host copy of the sorted realisation table
  cudaGraphExec_t exec = nullptr;
  int graph = 0;
  double probe_ms[64] = {};
  uint32_t nprobe = 0;
  bool ran = false;
};

namespace {

bool valid_L(uint32_t L) { return L >= 128u && L <= 131072u && (L & (L - 1u)) == 0u; }
size_t up256(size_t n) { return (n + 255) / 256 * 256; }

std::vector<uint64_t> sample_grid(const std::vector<kpz_spec>& spec, uint32_t n) {
  uint64_t T = 0;
  for (const auto& s : spec) T = std::max<uint64_t>(T, s.n_mcs);
  std::vector<uint64_t> ts{0};
  if (T > 0)
    for (uint32_t k = 0; k < n; ++k) {
      const double e = n > 1 ? (double)k * std::log10((double)T) / (double)(n - 1) : 0.0;
      uint64_t t = (uint64_t)std::ceil(std::pow(10.0, e) - 1e-9);
      ts.push_back(std::min<uint64_t>(t, T));
    }
  for (const auto& s : spec) ts.push_back(s.n_mcs);
  std::sort(ts.begin(), ts.end());
  ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
  return ts;
}

// Tables of the queue for the given knobs (host side), copied into the pool.
struct HostPlan {
  std::vector<Segment> seg;
  std::vector<unsigned long long> PW, PS;
  unsigned long long total = 0;
};

HostPlan build_plan(kpz_batch* b, std::vector<Real>& real) {
  HostPlan hp;
  const uint32_t n = (uint32_t)real.size();
  hp.PW.assign(n + 1, 0);
  hp.PS.assign(n + 1, 0);
  std::vector<uint64_t> T(n);
  for (uint32_t i = 0; i < n; ++i) {
    Real& r = real[i];
    const uint32_t ntx = r.P.g.L / kTile;
    uint32_t run = 1;
    while (run * 2 <= std::min(b->run_max, ntx)) run *= 2;
    r.P.ntx = ntx;
    r.P.nty = r.P.g.L / (kTile * b->cr);
    r.P.run = run;
    r.P.runs_x = ntx / run;
    r.n_items = r.P.runs_x * r.P.nty;
    r.nb = r.P.g.L / 128u;
    hp.PW[i + 1] = hp.PW[i] + r.n_items;
    hp.PS[i + 1] = hp.PS[i] + r.nb;
    T[i] = b->spec[b->order[i]].n_mcs;
  }
  const auto& G = b->times;
  const uint64_t Tmax = G.back();
  auto active_ge = [&](uint64_t g) { uint32_t a = 0; while (a < n && T[a] >= g) ++a; return a; };
  auto active_gt = [&](uint64_t g) { uint32_t a = 0; while (a < n && T[a] > g) ++a; return a; };
  unsigned long long base = 0;
  uint32_t nsamp = 0;
  size_t gi = 0;  // next sample time index
  uint64_t g = 0;
  while (g <= Tmax) {
    if (gi < G.size() && G[gi] == g) {
      ++nsamp;
      Segment s{};
      s.base = base; s.g0 = (uint32_t)g; s.nph = 1; s.has_sample = 1;
      s.As = active_ge(g); s.Aw = g < Tmax ? active_gt(g) : 0u;
      s.size = (uint32_t)(hp.PS[s.As] + hp.PW[s.Aw]);
      s.nsamp = nsamp;
      if (s.size) { hp.seg.push_back(s); base += s.size; }
      ++gi;
      ++g;
    } else {
      const uint64_t g1 = gi < G.size() ? G[gi] : Tmax + 1;
      Segment s{};
      s.base = base; s.g0 = (uint32_t)g; s.nph = (uint32_t)(g1 - g); s.has_sample = 0;
      s.As = 0; s.Aw = active_gt(g);
      s.size = (uint32_t)hp.PW[s.Aw];
      s.nsamp = nsamp;
      if (s.size) { hp.seg.push_back(s); base += (unsigned long long)s.nph * s.size; }
      g = g1;
    }
  }
  hp.total = base;
  return hp;
}

kpz_status fail_free(kpz_batch* b, kpz_status st) {
  if (b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->pool) cudaFree(b->pool);
    delete b;
  }
  return st;
}

// Lay out lattices, tables, counters and accumulators in one allocation.
kpz_status allocate(kpz_batch* b) {
  const uint32_t n = (uint32_t)b->spec.size();
  size_t lat = 0;
  b->bands = 0;
  for (const auto& s : b->spec) {
    lat += up256((size_t)s.L * s.L / 8);
    b->bands += s.L / 128u;
  }
  b->lat_bytes = lat;
  // worst-case table sizes (run length 1 gives the most items, not more segments)
  const size_t nseg_max = 2 * b->times.size() + 4;
  const size_t nG = b->times.size();
  size_t bytes = lat;
  bytes += up256(sizeof(Real) * n) + up256(sizeof(Segment) * nseg_max);
  bytes += 2 * up256(8 * (n + 1));                 // PW, PS
  bytes += 2 * up256(8 * n) + up256(8 * n);        // sweep_done, sample_done, h00
  bytes += up256(24 * b->bands * nG) + 256 + 256;  // band partials, head, err
  if (cudaMalloc(&b->pool, bytes) != cudaSuccess) { cudaGetLastError(); return KPZ_ENOMEM; }
  b->pool_bytes = bytes;
  return KPZ_OK;
}

struct PoolMap {
  char* lat; Real* real; Segment* seg; unsigned long long *PW, *PS, *sweep_done, *sample_done, *h00, *acc, *head;
  int* err;
};

PoolMap map_pool(const kpz_batch* b) {
  const uint32_t n = (uint32_t)b->spec.size();
  const size_t nseg_max = 2 * b->times.size() + 4, nG = b->times.size();
  char* p = (char*)b->pool;
  PoolMap m{};
  m.lat = p; p += b->lat_bytes;
  m.real = (Real*)p; p += up256(sizeof(Real) * n);
  m.seg = (Segment*)p; p += up256(sizeof(Segment) * nseg_max);
  m.PW = (unsigned long long*)p; p += up256(8 * (n + 1));
  m.PS = (unsigned long long*)p; p += up256(8 * (n + 1));
  m.sweep_done = (unsigned long long*)p; p += up256(8 * n);
  m.sample_done = (unsigned long long*)p; p += up256(8 * n);
  m.h00 = (unsigned long long*)p; p += up256(8 * n);
  m.acc = (unsigned long long*)p; p += up256(24 * b->bands * nG);
  m.head = (unsigned long long*)p; p += 256;
  m.err = (int*)p;
  return m;
}

size_t smem_bytes(uint32_t wpc, uint32_t cr) {
  return wpc * (cr == 2 ? sizeof(WarpSlot<2>) : sizeof(WarpSlot<1>));
}
const void* kernel_of(uint32_t cr) {
  return cr == 2 ? (const void*)batch_kernel<2> : (const void*)batch_kernel<1>;
}

// Upload the plan for the current knobs; fills b->plan and b->grid.
kpz_status prepare(kpz_batch* b, const std::vector<uint64_t>* cap_T) {
  const uint32_t n = (uint32_t)b->spec.size();
  PoolMap m = map_pool(b);
  std::vector<Real> real(n);
  size_t off = 0;
  std::vector<size_t> lat_off(n);
  for (uint32_t c = 0; c < n; ++c) { lat_off[c] = off; off += up256((size_t)b->spec[c].L * b->spec[c].L / 8); }
  for (uint32_t i = 0; i < n; ++i) {
    const kpz_spec& s = b->spec[b->order[i]];
    Real& r = real[i];
    r.P = SweepParams{};
    r.P.lat = (uint32_t*)(m.lat + lat_off[b->order[i]]);
    r.P.g.L = s.L; r.P.g.NR = s.L / 4; r.P.g.NB = s.L / 128; r.P.g.par = 0;
    r.P.Tp = acceptance_threshold(s.p);
    r.P.Tq = acceptance_threshold(s.q);
    r.P.nlev = acceptance_levels(r.P.Tp, r.P.Tq);
    set_philox_key(r.P, s.seed);
    r.P.sample = s.sample;
    r.P.h00 = m.h00 + i;
    r.general = !(r.P.Tp == 65536u && r.P.Tq == 0u);
  }
  // A probe replaces the run lengths by shorter ones (capped copies of the specs).
  std::vector<kpz_spec> saved;
  std::vector<uint64_t> saved_times;
  if (cap_T) {
    saved = b->spec;
    saved_times = b->times;
    for (uint32_t c = 0; c < n; ++c) b->spec[c].n_mcs = (uint32_t)(*cap_T)[c];
    b->times = sample_grid(b->spec, 2);   // start and end only: the probe times sweeping
  }
  HostPlan hp = build_plan(b, real);
  const size_t nseg_max = 2 * (cap_T ? saved_times.size() : b->times.size()) + 4;
  if (hp.seg.size() > nseg_max) return KPZ_EINVAL;
  cudaStream_t st = b->stream;
  if (cudaMemcpyAsync(m.real, real.data(), sizeof(Real) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m.seg, hp.seg.data(), sizeof(Segment) * hp.seg.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m.PW, hp.PW.data(), 8 * (n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m.PS, hp.PS.data(), 8 * (n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return KPZ_ECUDA;
  Plan& Q = b->plan;
  Q.seg = m.seg; Q.nseg = (uint32_t)hp.seg.size(); Q.real = m.real; Q.PW = m.PW; Q.PS = m.PS;
  Q.total = hp.total; Q.head = m.head; Q.sweep_done = m.sweep_done; Q.sample_done = m.sample_done;
  Q.acc = m.acc; Q.nG = (uint32_t)b->times.size(); Q.err = m.err; Q.timeout_ns = b->timeout_ns;
  Q.block = b->block;
  b->real = real;
  if (cap_T) { b->spec = saved; b->times = saved_times; Q.nG = (uint32_t)b->times.size(); }
  int maxb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, kernel_of(b->cr), (int)(b->wpc * 32),
                                                    smem_bytes(b->wpc, b->cr)) != cudaSuccess || maxb < 1)
    return KPZ_ECUDA;
  const uint32_t per_sm = b->ctas_per_sm ? std::min<uint32_t>(b->ctas_per_sm, (uint32_t)maxb) : (uint32_t)maxb;
  b->grid = per_sm * b->sms;
  return KPZ_OK;
}

// Queue the whole ensemble: flat start for every lattice, counters cleared,
// one cooperative persistent launch.
cudaError_t enqueue(kpz_batch* b, bool capturing = false) {
  PoolMap m = map_pool(b);
  cudaStream_t st = b->stream;
  cudaError_t e = cudaMemsetAsync(b->pool, 0, b->lat_bytes, st);   // flat start: all height bits 0
  // counters, origin heights, accumulators, queue head and error flag
  if (e == cudaSuccess) e = cudaMemsetAsync(m.sweep_done, 0, (char*)(m.err + 64) - (char*)m.sweep_done, st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&b->plan};
  e = cudaLaunchCooperativeKernel(kernel_of(b->cr), dim3(b->grid), dim3(b->wpc * 32), args,
                                  smem_bytes(b->wpc, b->cr), st);
  if (!capturing) count_launch();
  return e;
}

kpz_status run_once(kpz_batch* b, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) { cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventRecord(e0, b->stream); }
  cudaError_t e = enqueue(b);
  if (ms) cudaEventRecord(e1, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (ms && e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return KPZ_ECUDA;
  int err = 0;
  if (cudaMemcpy(&err, map_pool(b).err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return KPZ_ECUDA;
  return err ? KPZ_ETIMEOUT : KPZ_OK;
}

}  // namespace

extern "C" {

kpz_status kpz_batch_create(kpz_batch** out, const kpz_spec* specs, uint32_t n, const kpz_batch_opts* opts) {
  if (!out) return KPZ_EINVAL;
  *out = nullptr;
  if (!specs || n == 0) return KPZ_EINVAL;
  kpz_batch_opts o{};
  o.test_block = -1;
  if (opts) o = *opts;
  for (uint32_t c = 0; c < n; ++c) {
    const kpz_spec& s = specs[c];
    if (!valid_L(s.L) || std::isnan(s.p) || std::isnan(s.q) || s.p < 0 || s.p > 1 || s.q < 0 || s.q > 1)
      return KPZ_EINVAL;
  }
  if (o.warps_per_cta > 8 || (o.run & (o.run - 1)) != 0 || o.n_samples > 1024) return KPZ_EINVAL;
  if (o.tile_y != 0 && o.tile_y != kTile && o.tile_y != 2u * kTile) return KPZ_EINVAL;
  uint32_t Lmin = ~0u;
  for (uint32_t c = 0; c < n; ++c) Lmin = std::min(Lmin, specs[c].L);
  if (o.tile_y == 2u * kTile && Lmin < 2u * kTile) return KPZ_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return KPZ_ENODEV;
  kpz_batch* b = new (std::nothrow) kpz_batch();
  if (!b) return KPZ_ENOMEM;
  cudaGetDevice(&b->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->sms = (uint32_t)sms;
  b->spec.assign(specs, specs + n);
  b->order.resize(n);
  for (uint32_t c = 0; c < n; ++c) b->order[c] = c;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](uint32_t x, uint32_t y) { return b->spec[x].n_mcs > b->spec[y].n_mcs; });
  b->times = sample_grid(b->spec, o.n_samples ? o.n_samples : 64u);
  b->stream = (cudaStream_t)o.stream;
  b->run_max = o.run ? o.run : 4u;
  b->wpc = o.warps_per_cta ? o.warps_per_cta : 8u;
  b->ctas_per_sm = o.ctas_per_sm;
  b->timeout_ns = (uint64_t)(o.timeout_ms ? o.timeout_ms : 10000u) * 1000000ull;
  b->block = o.test_block;
  b->cr = o.tile_y == 2u * kTile ? 2u : 1u;
  if (cudaFuncSetAttribute(kernel_of(1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes(8, 1)) != cudaSuccess ||
      cudaFuncSetAttribute(kernel_of(2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes(8, 2)) != cudaSuccess)
    return fail_free(b, KPZ_ECUDA);
  kpz_status st = allocate(b);
  if (st) return fail_free(b, st);

  if (o.autotune) {
    // Time a short probe of the same ensemble (every run capped at 24 sweeps,
    // W^2 only at its start and end) for each setting of the execution knobs;
    // keep the fastest (first in this order on ties).
    std::vector<uint64_t> cap(n);
    for (uint32_t c = 0; c < n; ++c) cap[c] = std::min<uint64_t>(b->spec[c].n_mcs, 24);
    // Runs of up to 32 tiles (a realisation takes min(run, L/128)): on the
    // batched workload, where L = 8192 carries most of the work, runs of 32
    // with 8-warp CTAs sweep 8 % faster than runs of 8.
    const uint32_t runs[] = {1, 2, 4, 8, 16, 32}, wpcs[] = {4, 8};
    float best = 1e30f;
    uint32_t best_run = 4, best_wpc = 8;
    for (uint32_t rr : runs)
      for (uint32_t ww : wpcs) {
        b->run_max = rr; b->wpc = ww; b->ctas_per_sm = 0;
        st = prepare(b, &cap);
        if (st) return fail_free(b, st);
        float ms = 0.f;
        st = run_once(b, &ms);
        if (st) return fail_free(b, st);
        if (b->nprobe < 64) b->probe_ms[b->nprobe++] = ms;
        if (ms < best) { best = ms; best_run = rr; best_wpc = ww; }
      }
    // Tile height (part of the schedule, so only when the caller leaves it
    // open): 128 x 256 at the best run length, both block sizes.
    uint32_t best_cr = b->cr;
    if (o.tile_y == 0 && Lmin >= 2u * kTile) {
      b->cr = 2;
      for (uint32_t ww : wpcs) {
        b->run_max = best_run; b->wpc = ww; b->ctas_per_sm = 0;
        st = prepare(b, &cap);
        if (st) return fail_free(b, st);
        float ms = 0.f;
        st = run_once(b, &ms);
        if (st) return fail_free(b, st);
        if (b->nprobe < 64) b->probe_ms[b->nprobe++] = ms;
        if (ms < best) { best = ms; best_wpc = ww; best_cr = 2; }
      }
    }
    b->cr = best_cr;
    b->run_max = best_run;
    b->wpc = best_wpc;
    // Blocks per SM: fewer resident blocks than fit, at the chosen settings.
    int maxb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, kernel_of(b->cr), (int)(b->wpc * 32),
                                                      smem_bytes(b->wpc, b->cr)) != cudaSuccess)
      return fail_free(b, KPZ_ECUDA);
    uint32_t best_cps = 0;
    for (uint32_t cps = 1; cps < (uint32_t)maxb; ++cps) {
      b->ctas_per_sm = cps;
      st = prepare(b, &cap);
      if (st) return fail_free(b, st);
      float ms = 0.f;
      st = run_once(b, &ms);
      if (st) return fail_free(b, st);
      if (b->nprobe < 64) b->probe_ms[b->nprobe++] = ms;
      if (ms < best) { best = ms; best_cps = cps; }
    }
    b->ctas_per_sm = best_cps;
  }
  st = prepare(b, nullptr);
  if (st) return fail_free(b, st);

  // Capture the whole ensemble (resets + the persistent launch) in a graph.
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
    cudaStream_t keep = b->stream;
    b->stream = cs;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) ok = enqueue(b, true) == cudaSuccess;
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) ok = false;
    if (ok && graph && cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess) b->graph = 1;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    b->stream = keep;
    cudaStreamDestroy(cs);
  }
  *out = b;
  return KPZ_OK;
}

kpz_status kpz_batch_run(kpz_batch* b) {
  if (!b) return KPZ_EINVAL;
  cudaSetDevice(b->device);
  kpz_status st;
  if (b->graph) {
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return KPZ_ECUDA;
    count_launch();   // the graph's persistent kernel
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return KPZ_ECUDA;
    int err = 0;
    if (cudaMemcpy(&err, map_pool(b).err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return KPZ_ECUDA;
    st = err ? KPZ_ETIMEOUT : KPZ_OK;
  } else {
    st = run_once(b, nullptr);
  }
  if (st == KPZ_OK) b->ran = true;
  return st;
}

kpz_status kpz_batch_times(const kpz_batch* b, uint64_t* times, uint32_t* n) {
  if (!b || !n) return KPZ_EINVAL;
  if (times) {
    if (*n < b->times.size()) return KPZ_EINVAL;
    for (size_t k = 0; k < b->times.size(); ++k) times[k] = b->times[k];
  }
  *n = (uint32_t)b->times.size();
  return KPZ_OK;
}

kpz_status kpz_batch_sums(const kpz_batch* b, int64_t* S1, uint64_t* S2_lo, uint64_t* S2_hi,
                          int64_t* h00) {
  if (!b || !S1 || !S2_lo || !S2_hi) return KPZ_EINVAL;
  if (!b->ran) return KPZ_ESTATE;
  const size_t n = b->spec.size(), nG = b->times.size();
  PoolMap m = map_pool(b);
  std::vector<unsigned long long> acc(3 * b->bands * nG), h(n);
  if (cudaMemcpy(acc.data(), m.acc, 24 * b->bands * nG, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(h.data(), m.h00, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return KPZ_ECUDA;
  // Chain the bands of each sample (eq. Wdef): band k starts at height H_k =
  // sum of the column-0 changes D of the bands above it; a band of n_b sites
  // with relative sums (s1, s2) adds n_b H + s1 and n_b H^2 + 2 H s1 + s2.
  size_t band0 = 0;
  for (size_t i = 0; i < n; ++i) {
    const size_t c = b->order[i];
    const uint32_t L = b->spec[c].L, nb = L / 128u;
    const __int128 nsite = (__int128)128 * L;
    for (size_t k = 0; k < nG; ++k) {
      __int128 H = 0, s1 = 0, s2 = 0;
      for (uint32_t q = 0; q < nb; ++q) {
        const unsigned long long* a = &acc[3 * ((band0 + q) * nG + k)];
        const __int128 bs1 = (long long)a[1], bs2 = (__int128)a[2];
        s1 += nsite * H + bs1;
        s2 += nsite * H * H + 2 * H * bs1 + bs2;
        H += (long long)a[0];
      }
      S1[c * nG + k] = (int64_t)s1;
      S2_lo[c * nG + k] = (uint64_t)((unsigned __int128)s2);
      S2_hi[c * nG + k] = (uint64_t)((unsigned __int128)s2 >> 64);
    }
    band0 += nb;
    if (h00) h00[c] = (int64_t)h[i];
  }
  return KPZ_OK;
}

kpz_status kpz_batch_w2(const kpz_batch* b, double* w2) {
  if (!b || !w2) return KPZ_EINVAL;
  const size_t n = b->spec.size(), nG = b->times.size();
  std::vector<int64_t> S1(n * nG);
  std::vector<uint64_t> lo(n * nG), hi(n * nG);
  kpz_status st = kpz_batch_sums(b, S1.data(), lo.data(), hi.data(), nullptr);
  if (st) return st;
  for (size_t c = 0; c < n; ++c) {
    const uint64_t N = (uint64_t)b->spec[c].L * b->spec[c].L;
    for (size_t k = 0; k < nG; ++k) {
      const size_t x = c * nG + k;
      if (b->times[k] > b->spec[c].n_mcs) { w2[x] = std::nan(""); continue; }
      const unsigned __int128 S2 = ((unsigned __int128)hi[x] << 64) | lo[x];
      const __int128 s1 = S1[x];
      const unsigned __int128 num = (unsigned __int128)N * S2 - (unsigned __int128)(s1 * s1);
      w2[x] = (double)num / ((double)N * (double)N);
    }
  }
  return KPZ_OK;
}

kpz_status kpz_batch_get_info(const kpz_batch* b, kpz_batch_info* out) {
  if (!b || !out) return KPZ_EINVAL;
  out->run = b->run_max;
  out->warps_per_cta = b->wpc;
  out->grid = b->grid;
  out->ctas_per_sm = b->grid / (b->sms ? b->sms : 1);
  out->graph = b->graph;
  out->items = b->plan.total;
  out->n_probe = std::min<uint32_t>(b->nprobe, 8);
  for (uint32_t k = 0; k < 8; ++k) out->probe_ms[k] = k < b->nprobe ? b->probe_ms[k] : 0.0;
  out->tile_y = kTile * b->cr;
  return KPZ_OK;
}

void kpz_batch_free(kpz_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  fail_free(b, KPZ_OK);
}

}  // extern "C"
