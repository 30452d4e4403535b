// kpz_api.cu -- the C ABI declared in include/kpz.h: argument checks, device
// memory, stream handling and the host side of each call. All lattice
// arithmetic runs in the kernels of kpz_sweep.cu and kpz_observe.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <string>

#include "kpz.h"
#include "kpz_internal.h"
#include "kpz_rsu.h"

using namespace kpz;

namespace kpz {
static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace kpz

struct kpz_ctx {
  Geometry g{};
  uint32_t Tp = 0, Tq = 0, nlev = 0, sample = 0;
  double p = 0.0, q = 0.0;             // as given to kpz_init (checkpoint header)
  uint64_t seed = 0;
  uint32_t run = 1, wpc = 8;
  uint32_t tile_y = 128;               // tile height in sites (128 or 256)
  uint32_t decomposition = 0;          // device layer: 0 dead border, 1 tile sets
  uint32_t cell = 4;                   // work-group cell edge: 4 or 2
  uint32_t colour_m = 3;               // decomposition 2: subset sparsity
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_buf = false;
  void* buf = nullptr;
  void* rsu_scratch = nullptr;         // decomposition 4: per-sweep attempt buckets
  size_t buf_bytes = 0;
  uint32_t* lat = nullptr;             // L*L/32 words (one bit per site)
  uint64_t* t_dev = nullptr;           // sweep counter
  unsigned long long* h00 = nullptr;   // absolute height of site (0,0)
  unsigned long long* acc = nullptr;   // S1, S2 lo, S2 hi
  uint32_t* hcar = nullptr;            // import: height of (0, j0) modulo 4
  uint32_t* queue = nullptr;           // sweep work queue (zero between launches)
  int32_t* col0 = nullptr;             // h(0,j)
  void* io = nullptr;                  // staging band for host transfers
  size_t io_bytes = 0;
  // Slope import/export: copies on io_stream overlap the conversion kernels
  // on `stream`, the staging band split into two halves. Events: [0..1] half
  // filled (copy done / kernel done), [2..3] half free, [4] stream -> io_stream.
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev[5] = {};
  uint64_t t_host = 0;
  bool poisoned = false;
  std::string err;
};

namespace {

constexpr size_t kAlign = 256;
// Staging band for host transfers: the packed slope array (L^2/4 bytes) up to
// 64 MiB. A slope import or export streams through its two halves, each copy
// overlapping the conversion kernel of the other half; checkpoint file I/O
// goes through a host buffer of the same size at most.
constexpr size_t kIoMax = size_t(64) << 20;
constexpr size_t kCkptHostMax = kIoMax;

size_t align_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// Largest lattice: 2^18 (8 GiB at one bit per site, plus 65 MiB of scratch).
bool valid_L(uint32_t L) { return L >= 128u && L <= 262144u && (L & (L - 1u)) == 0u; }

struct Layout {
  size_t lat, small, col0, io, total;
};

Layout layout(uint32_t L) {
  Layout y{};
  const size_t lat_bytes = (size_t)L * L / 8;   // 1 bit per site
  y.lat = 0;
  y.small = align_up(lat_bytes);                 // t, h00, acc[3], hcar, queue
  y.col0 = y.small + kAlign;
  y.io = y.col0 + align_up((size_t)L * 4);
  const size_t io_bytes = std::min(kIoMax, (size_t)L * L / 4);
  y.total = y.io + align_up(io_bytes);
  return y;
}


kpz_status fail(kpz_ctx* c, kpz_status st, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (st == KPZ_ECUDA || st == KPZ_ETIMEOUT) c->poisoned = true;
  }
  return st;
}

kpz_status cuda_fail(kpz_ctx* c, cudaError_t e, const char* what) {
  return fail(c, KPZ_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define KPZ_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);    \
  } while (0)

kpz_status enter(kpz_ctx* ctx) {
  if (!ctx) return KPZ_EINVAL;
  if (ctx->poisoned) return KPZ_ESTATE;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return KPZ_OK;
}

// Creates the copy stream and events on first use and orders io_stream after
// the work already queued on the context's stream.
cudaError_t io_prepare(kpz_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (!c->io_stream) {
    // All or nothing: on failure nothing is kept and the next call tries again.
    cudaStream_t s = nullptr;
    cudaEvent_t ev[5] = {};
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
      if (s) cudaStreamDestroy(s);
      return e;
    }
    c->io_stream = s;
    for (int i = 0; i < 5; ++i) c->io_ev[i] = ev[i];
  }
  e = cudaEventRecord(c->io_ev[4], c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->io_stream, c->io_ev[4], 0);
  return e;
}

// Rows per band when the staging band is used as two halves.
uint32_t io_band_rows(const kpz_ctx* c, size_t row_bytes, size_t* half) {
  *half = (c->io_bytes / 2) / kAlign * kAlign;
  return (uint32_t)std::min<size_t>(c->g.L, *half / row_bytes) & ~3u;
}

SweepParams sweep_params(const kpz_ctx* c) {
  SweepParams P{};
  P.lat = c->lat;
  P.t_dev = c->t_dev;
  P.g = c->g;
  P.ntx = c->g.L / kTile;
  P.nty = c->g.L / c->tile_y;
  P.run = c->run;
  P.runs_x = P.ntx / c->run;
  P.Tp = c->Tp;
  P.Tq = c->Tq;
  P.nlev = c->nlev;
  set_philox_key(P, c->seed);
  P.sample = c->sample;
  P.h00 = c->h00;
  P.queue = c->queue;
  P.cell = c->cell;
  return P;
}


}  // namespace

extern "C" {

uint64_t kpz_launch_count(void) { return kpz::g_launches.load(std::memory_order_relaxed); }

size_t kpz_device_bytes(uint32_t L) { return valid_L(L) ? layout(L).total : 0; }

const char* kpz_strerror(kpz_status st) {
  switch (st) {
    case KPZ_OK: return "ok";
    case KPZ_EINVAL: return "invalid argument";
    case KPZ_ENOMEM: return "out of device memory";
    case KPZ_ECUDA: return "CUDA error";
    case KPZ_ETIMEOUT: return "device wait timed out";
    case KPZ_ESTATE: return "context poisoned by an earlier error";
    case KPZ_ENODEV: return "no CUDA device";
    case KPZ_ERANGE: return "lattice larger than the 131072 maximum of the static scratch";
    case KPZ_ECKPT: return "checkpoint file unreadable, truncated or corrupt";
  }
  return "unknown status";
}

const char* kpz_last_error(const kpz_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

kpz_status kpz_init(kpz_ctx** out, uint32_t L, double p, double q, uint64_t seed, uint32_t sample,
                    int init, const kpz_opts* opts) {
  if (!out) return KPZ_EINVAL;
  *out = nullptr;
  if (!valid_L(L) || std::isnan(p) || std::isnan(q) || p < 0.0 || p > 1.0 || q < 0.0 || q > 1.0 ||
      init != 0)
    return KPZ_EINVAL;
  kpz_opts o{};
  if (opts) o = *opts;
  if (o.decomposition > 4u || (o.decomposition == 1u && ((o.by != 0 && o.by != kTile) || L < 2u * kTile)) ||
      (o.decomposition == 4u && L > 8192u) ||
      (o.decomposition >= 2u && ((o.by != 0 && o.by != kTile) || (o.cell != 0 && o.cell != 4u))) ||
      o.colour_sparsity > 4u || (o.colour_sparsity != 0 && o.decomposition != 2u))
    return KPZ_EINVAL;
  if ((o.cell != 0 && o.cell != 4u && o.cell != 2u) ||
      (o.cell == 2u && (o.decomposition != 0u || (o.by != 0 && o.by != kTile))))
    return KPZ_EINVAL;
  if ((o.bx != 0 && o.bx != kTile) ||
      (o.by != 0 && o.by != kTile && !(o.by == 2u * kTile && L >= 2u * kTile)))
    return KPZ_EINVAL;
  const uint32_t ntx = L / kTile;
  if (o.run != 0 && ((o.run & (o.run - 1)) != 0 || o.run > ntx)) return KPZ_EINVAL;
  if (o.warps_per_cta > 8) return KPZ_EINVAL;
  const Layout y = layout(L);
  if (o.dev_buf && (o.dev_bytes < y.total || ((uintptr_t)o.dev_buf % kAlign) != 0)) return KPZ_EINVAL;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return KPZ_ENODEV;

  kpz_ctx* ctx = new (std::nothrow) kpz_ctx();
  if (!ctx) return KPZ_ENOMEM;
  cudaGetDevice(&ctx->device);
  ctx->g.L = L;
  ctx->g.NR = L / 4;
  ctx->g.NB = L / 128;
  ctx->g.par = 0;
  ctx->p = p;
  ctx->q = q;
  ctx->Tp = acceptance_threshold(p);
  ctx->Tq = acceptance_threshold(q);
  ctx->nlev = acceptance_levels(ctx->Tp, ctx->Tq);
  ctx->seed = seed;
  ctx->sample = sample;
  ctx->tile_y = o.by ? o.by : kTile;
  ctx->decomposition = o.decomposition;
  ctx->cell = o.cell ? o.cell : 4u;
  ctx->colour_m = o.colour_sparsity ? o.colour_sparsity : 3u;
  // Default schedule, measured on GB300 at p = 1 (results do not depend on
  // it): runs of 8 tiles and 8-warp CTAs up to 256 tiles per row; from 512
  // tiles per row runs of ntx/32 tiles, which halve the per-run cost (window
  // prologue, start copy, edge write-backs) while about 4.5 (L = 2^16) or 9
  // (L = 2^17) runs per resident warp keep the last wave short, with 4-warp
  // CTAs for 128-row tiles. L = 2^16: 0.4765 ms per sweep against 0.4954 ms;
  // L = 2^17: 1.827 ms against 1.920 ms.
  const bool wide = ntx >= 512u;
  ctx->run = o.run ? o.run : (wide ? ntx / 32u : std::min(8u, ntx));   // tiles per work-queue chunk
  ctx->wpc = o.warps_per_cta ? o.warps_per_cta : (wide && ctx->tile_y == kTile ? 4u : 8u);
  ctx->stream = (cudaStream_t)o.stream;
  if (o.dev_buf) {
    ctx->buf = o.dev_buf;
    ctx->buf_bytes = o.dev_bytes;
  } else {
    cudaError_t e = cudaMalloc(&ctx->buf, y.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return KPZ_ENOMEM;
    }
    ctx->own_buf = true;
    ctx->buf_bytes = y.total;
  }
  if (ctx->decomposition == 4u) {   // per-sweep attempt buckets of the exact random-sequential sweep
    cudaError_t e = cudaMalloc(&ctx->rsu_scratch, rsu_scratch_bytes(L));
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ctx->own_buf) cudaFree(ctx->buf);
      delete ctx;
      return KPZ_ENOMEM;
    }
  }
  char* base = (char*)ctx->buf;
  ctx->lat = (uint32_t*)(base + y.lat);
  ctx->t_dev = (uint64_t*)(base + y.small);
  ctx->h00 = (unsigned long long*)(base + y.small + 8);
  ctx->acc = (unsigned long long*)(base + y.small + 16);
  ctx->hcar = (uint32_t*)(base + y.small + 40);
  ctx->queue = (uint32_t*)(base + y.small + 48);
  ctx->col0 = (int32_t*)(base + y.col0);
  ctx->io = base + y.io;
  ctx->io_bytes = y.total - y.io;

  kpz_status st = KPZ_OK;
  cudaError_t e = cudaMemsetAsync(base + y.small, 0, kAlign, ctx->stream);
  if (e == cudaSuccess) e = launch_init_flat(ctx->lat, ctx->g, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) st = cuda_fail(ctx, e, "kpz_init");
  *out = ctx;
  return st;
}

kpz_status kpz_reset(kpz_ctx* ctx) {
  kpz_status st = enter(ctx);
  if (st) return st;
  KPZ_CUDA(cudaMemsetAsync(ctx->t_dev, 0, 2 * sizeof(uint64_t), ctx->stream));
  KPZ_CUDA(launch_init_flat(ctx->lat, ctx->g, ctx->stream));
  ctx->t_host = 0;
  ctx->g.par = 0;
  return KPZ_OK;
}

kpz_status kpz_run(kpz_ctx* ctx, uint64_t n_mcs) {
  kpz_status st = enter(ctx);
  if (st) return st;
  SweepParams P = sweep_params(ctx);
  while (n_mcs > 0) {
    const uint32_t chunk = (uint32_t)std::min<uint64_t>(n_mcs, 1u << 20);
    for (uint32_t i = 0; i < chunk; ++i) {
      P.s_add = i;
      if (ctx->decomposition == 1u)      KPZ_CUDA(launch_sweep_tilesets(P, ctx->stream));
      else if (ctx->decomposition == 2u) KPZ_CUDA(launch_sweep_colour(P, ctx->colour_m, ctx->stream));
      else if (ctx->decomposition == 3u) KPZ_CUDA(launch_sweep_db2(P, ctx->stream));
      else if (ctx->decomposition == 4u) KPZ_CUDA(launch_sweep_rsu(P, ctx->rsu_scratch, ctx->stream));
      else                               KPZ_CUDA(launch_sweep(P, ctx->wpc, ctx->stream));
    }
    KPZ_CUDA(launch_advance(ctx->t_dev, chunk, ctx->stream));
    ctx->t_host += chunk;
    n_mcs -= chunk;
  }
  return KPZ_OK;
}

kpz_status kpz_roughness(kpz_ctx* ctx, kpz_rough* out) {
  kpz_status st = enter(ctx);
  if (st) return st;
  if (!out) return fail(ctx, KPZ_EINVAL, "null output");
  KPZ_CUDA(launch_roughness(ctx->lat, ctx->g, ctx->col0, ctx->acc, ctx->stream));
  unsigned long long host[4];
  KPZ_CUDA(cudaMemcpyAsync(host, ctx->acc, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           ctx->stream));
  KPZ_CUDA(cudaMemcpyAsync(host + 3, ctx->h00, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           ctx->stream));
  KPZ_CUDA(cudaStreamSynchronize(ctx->stream));
  const uint64_t N = (uint64_t)ctx->g.L * ctx->g.L;
  out->t_mcs = ctx->t_host;
  out->n_sites = N;
  out->sum_h = (int64_t)host[0];
  out->sum_h2_lo = host[1];
  out->sum_h2_hi = host[2];
  out->h00 = (int64_t)host[3];
  const unsigned __int128 S2 = ((unsigned __int128)host[2] << 64) | host[1];
  const __int128 S1 = (int64_t)host[0];
  const unsigned __int128 num = (unsigned __int128)N * S2 - (unsigned __int128)(S1 * S1);
  out->w2 = (double)num / ((double)N * (double)N);
  return KPZ_OK;
}

kpz_status kpz_heights(kpz_ctx* ctx, int64_t* host_out, int absolute) {
  kpz_status st = enter(ctx);
  if (st) return st;
  if (!host_out) return fail(ctx, KPZ_EINVAL, "null output");
  const uint32_t L = ctx->g.L;
  KPZ_CUDA(launch_col0(ctx->lat, ctx->g, ctx->col0, ctx->stream));
  const uint32_t band = (uint32_t)std::max<size_t>(1, std::min<size_t>(L, ctx->io_bytes / ((size_t)L * 8)));
  for (uint32_t j0 = 0; j0 < L; j0 += band) {
    const uint32_t nr = std::min(band, L - j0);
    KPZ_CUDA(launch_heights(ctx->lat, ctx->g, ctx->col0, j0, nr, absolute ? ctx->h00 : nullptr,
                            (int64_t*)ctx->io, ctx->stream));
    KPZ_CUDA(cudaMemcpyAsync(host_out + (size_t)j0 * L, ctx->io, (size_t)nr * L * 8,
                             cudaMemcpyDeviceToHost, ctx->stream));
    KPZ_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return KPZ_OK;
}

kpz_status kpz_slopes(kpz_ctx* ctx, uint32_t* host_out) {
  kpz_status st = enter(ctx);
  if (st) return st;
  if (!host_out) return fail(ctx, KPZ_EINVAL, "null output");
  const uint32_t L = ctx->g.L;
  const size_t row_bytes = (size_t)L / 16 * 4;
  size_t half = 0;
  const uint32_t band = io_band_rows(ctx, row_bytes, &half);
  char* buf[2] = {(char*)ctx->io, (char*)ctx->io + half};
  KPZ_CUDA(io_prepare(ctx));
  uint32_t b = 0;
  for (uint32_t j0 = 0; j0 < L; j0 += band, ++b) {
    const uint32_t nr = std::min(band, L - j0), k = b & 1u;
    if (b >= 2) KPZ_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->io_ev[2 + k], 0));   // half k read out
    KPZ_CUDA(launch_export_packed(ctx->lat, ctx->g, j0, nr, (uint32_t*)buf[k], ctx->stream));
    KPZ_CUDA(cudaEventRecord(ctx->io_ev[k], ctx->stream));
    KPZ_CUDA(cudaStreamWaitEvent(ctx->io_stream, ctx->io_ev[k], 0));
    KPZ_CUDA(cudaMemcpyAsync((char*)host_out + (size_t)j0 * row_bytes, buf[k], nr * row_bytes,
                             cudaMemcpyDeviceToHost, ctx->io_stream));
    KPZ_CUDA(cudaEventRecord(ctx->io_ev[2 + k], ctx->io_stream));
  }
  KPZ_CUDA(cudaStreamSynchronize(ctx->io_stream));
  return KPZ_OK;
}

kpz_status kpz_set_slopes(kpz_ctx* ctx, const uint32_t* host_in, int64_t h00, uint64_t t_mcs) {
  kpz_status st = enter(ctx);
  if (st) return st;
  if (!host_in) return fail(ctx, KPZ_EINVAL, "null input");
  const uint32_t L = ctx->g.L;
  const size_t row_bytes = (size_t)L / 16 * 4;
  size_t half = 0;
  const uint32_t band = io_band_rows(ctx, row_bytes, &half);
  char* buf[2] = {(char*)ctx->io, (char*)ctx->io + half};
  ctx->g.par = (uint32_t)(h00 & 1);
  const uint32_t h00_mod4 = (uint32_t)(h00 & 3);
  KPZ_CUDA(cudaMemcpyAsync(ctx->hcar, &h00_mod4, sizeof(uint32_t), cudaMemcpyHostToDevice,
                           ctx->stream));
  KPZ_CUDA(io_prepare(ctx));
  uint32_t b = 0;
  for (uint32_t j0 = 0; j0 < L; j0 += band, ++b) {
    const uint32_t nr = std::min(band, L - j0), k = b & 1u;
    if (b >= 2) KPZ_CUDA(cudaStreamWaitEvent(ctx->io_stream, ctx->io_ev[2 + k], 0));   // half k converted
    KPZ_CUDA(cudaMemcpyAsync(buf[k], (const char*)host_in + (size_t)j0 * row_bytes, nr * row_bytes,
                             cudaMemcpyHostToDevice, ctx->io_stream));
    KPZ_CUDA(cudaEventRecord(ctx->io_ev[k], ctx->io_stream));
    KPZ_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->io_ev[k], 0));
    KPZ_CUDA(launch_import_packed(ctx->lat, ctx->g, j0, nr, (const uint32_t*)buf[k], ctx->hcar,
                                  ctx->col0, ctx->stream));
    KPZ_CUDA(cudaEventRecord(ctx->io_ev[2 + k], ctx->stream));
  }
  unsigned long long small[2] = {(unsigned long long)t_mcs, (unsigned long long)h00};
  KPZ_CUDA(cudaMemcpyAsync(ctx->t_dev, small, sizeof(small), cudaMemcpyHostToDevice, ctx->stream));
  KPZ_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->t_host = t_mcs;
  return KPZ_OK;
}

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version, L;
  double p, q;
  uint32_t Tp, Tq;
  uint64_t seed;
  uint32_t sample, bx, by, decomposition;
  uint64_t t_mcs;
  int64_t h00;
};
static_assert(sizeof(CkptHeader) % 8 == 0, "checksum runs over 64-bit words");
constexpr char kCkptMagic[8] = {'K', 'P', 'Z', 'C', 'K', 'P', 'T', '1'};
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;

// FNV-1a over little-endian 64-bit words (n a multiple of 8).
uint64_t fnv_words(uint64_t h, const void* data, size_t n) {
  const unsigned char* b = (const unsigned char*)data;
  for (size_t i = 0; i < n; i += 8) {
    uint64_t w = 0;
    for (int k = 7; k >= 0; --k) w = (w << 8) | b[i + k];
    h = (h ^ w) * kFnvPrime;
  }
  return h;
}

struct File {
  FILE* f = nullptr;
  ~File() { if (f) fclose(f); }
};

}  // namespace

kpz_status kpz_ckpt_save(kpz_ctx* ctx, const char* path) {
  kpz_status st = enter(ctx);
  if (st) return st;
  if (!path) return fail(ctx, KPZ_EINVAL, "null path");
  const uint32_t L = ctx->g.L;
  CkptHeader hd{};
  memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.L = L;
  hd.p = ctx->p;
  hd.q = ctx->q;
  hd.Tp = ctx->Tp;
  hd.Tq = ctx->Tq;
  hd.seed = ctx->seed;
  hd.sample = ctx->sample;
  hd.bx = kTile;
  hd.by = ctx->tile_y;
  // bits 0-7: device layer, bit 8: C = 2, bits 12-15: colour sparsity (decomposition 2)
  hd.decomposition = ctx->decomposition | (ctx->cell == 2u ? 0x100u : 0u) |
                     (ctx->decomposition == 2u ? ctx->colour_m << 12 : 0u);
  unsigned long long small[2];
  KPZ_CUDA(cudaMemcpyAsync(small, ctx->t_dev, sizeof(small), cudaMemcpyDeviceToHost, ctx->stream));
  KPZ_CUDA(cudaStreamSynchronize(ctx->stream));
  hd.t_mcs = small[0];
  hd.h00 = (int64_t)small[1];
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) return fail(ctx, KPZ_ECKPT, std::string("cannot create ") + path);
  uint64_t h = fnv_words(kFnvBasis, &hd, sizeof(hd));
  if (fwrite(&hd, sizeof(hd), 1, out.f) != 1) return fail(ctx, KPZ_ECKPT, "write failed");
  const size_t row_bytes = (size_t)L / 16 * 4;
  const uint32_t band = (uint32_t)std::min<size_t>(L, std::min(ctx->io_bytes, kCkptHostMax) / row_bytes) & ~3u;
  std::string host((size_t)band * row_bytes, '\0');
  for (uint32_t j0 = 0; j0 < L; j0 += band) {
    const uint32_t nr = std::min(band, L - j0);
    KPZ_CUDA(launch_export_packed(ctx->lat, ctx->g, j0, nr, (uint32_t*)ctx->io, ctx->stream));
    KPZ_CUDA(cudaMemcpyAsync(&host[0], ctx->io, nr * row_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    KPZ_CUDA(cudaStreamSynchronize(ctx->stream));
    h = fnv_words(h, host.data(), nr * row_bytes);
    if (fwrite(host.data(), 1, nr * row_bytes, out.f) != nr * row_bytes)
      return fail(ctx, KPZ_ECKPT, "write failed");
  }
  if (fwrite(&h, sizeof(h), 1, out.f) != 1 || fflush(out.f) != 0)
    return fail(ctx, KPZ_ECKPT, "write failed");
  return KPZ_OK;
}

kpz_status kpz_ckpt_load(kpz_ctx** out, const char* path, const kpz_opts* opts) {
  if (!out || !path) return KPZ_EINVAL;
  *out = nullptr;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return KPZ_ECKPT;
  CkptHeader hd{};
  if (fread(&hd, sizeof(hd), 1, in.f) != 1 || memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1 ||
      !valid_L(hd.L) || hd.bx != kTile || (hd.by != kTile && hd.by != 2u * kTile) ||
      acceptance_threshold(hd.p) != hd.Tp || acceptance_threshold(hd.q) != hd.Tq || (hd.decomposition & ~0xF100u) > 4u)
    return KPZ_ECKPT;
  kpz_opts o{};
  if (opts) o = *opts;
  if ((o.bx != 0 && o.bx != hd.bx) || (o.by != 0 && o.by != hd.by)) return KPZ_EINVAL;
  const uint32_t dec = hd.decomposition & 0xFFu, cell = (hd.decomposition & 0x100u) ? 2u : 4u;
  const uint32_t cm = (hd.decomposition >> 12) & 0xFu;
  if ((o.decomposition != 0 && o.decomposition != dec) || (o.cell != 0 && o.cell != cell) ||
      (o.colour_sparsity != 0 && o.colour_sparsity != cm))
    return KPZ_EINVAL;
  o.colour_sparsity = dec == 2u ? cm : 0u;
  o.bx = hd.bx;
  o.by = hd.by;
  o.decomposition = dec;
  o.cell = cell;
  kpz_ctx* ctx = nullptr;
  kpz_status st = kpz_init(&ctx, hd.L, hd.p, hd.q, hd.seed, hd.sample, 0, &o);
  if (st) return st;
  auto bail = [&](kpz_status s) { kpz_free(ctx); return s; };
  uint64_t h = fnv_words(kFnvBasis, &hd, sizeof(hd));
  const uint32_t L = hd.L;
  const size_t row_bytes = (size_t)L / 16 * 4;
  const uint32_t band = (uint32_t)std::min<size_t>(L, std::min(ctx->io_bytes, kCkptHostMax) / row_bytes) & ~3u;
  std::string host((size_t)band * row_bytes, '\0');
  ctx->g.par = (uint32_t)(hd.h00 & 1);
  const uint32_t h00_mod4 = (uint32_t)(hd.h00 & 3);
  if (cudaMemcpyAsync(ctx->hcar, &h00_mod4, sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream) !=
      cudaSuccess)
    return bail(KPZ_ECUDA);
  for (uint32_t j0 = 0; j0 < L; j0 += band) {
    const uint32_t nr = std::min(band, L - j0);
    if (fread(&host[0], 1, nr * row_bytes, in.f) != nr * row_bytes) return bail(KPZ_ECKPT);
    h = fnv_words(h, host.data(), nr * row_bytes);
    if (cudaMemcpyAsync(ctx->io, host.data(), nr * row_bytes, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        launch_import_packed(ctx->lat, ctx->g, j0, nr, (const uint32_t*)ctx->io, ctx->hcar, ctx->col0,
                             ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      return bail(KPZ_ECUDA);
  }
  uint64_t want = 0;
  if (fread(&want, sizeof(want), 1, in.f) != 1 || want != h || fgetc(in.f) != EOF) return bail(KPZ_ECKPT);
  unsigned long long small[2] = {(unsigned long long)hd.t_mcs, (unsigned long long)hd.h00};
  if (cudaMemcpyAsync(ctx->t_dev, small, sizeof(small), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return bail(KPZ_ECUDA);
  ctx->t_host = hd.t_mcs;
  *out = ctx;
  return KPZ_OK;
}

kpz_status kpz_device_lattice(kpz_ctx* ctx, void** dev_ptr, size_t* bytes) {
  if (!ctx || !dev_ptr || !bytes) return KPZ_EINVAL;
  *dev_ptr = ctx->lat;
  *bytes = (size_t)ctx->g.L * ctx->g.L / 8;
  return KPZ_OK;
}

void kpz_free(kpz_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->io_stream) {
    cudaStreamSynchronize(ctx->io_stream);
    for (cudaEvent_t ev : ctx->io_ev)
      if (ev) cudaEventDestroy(ev);
    cudaStreamDestroy(ctx->io_stream);
  }
  if (ctx->own_buf && ctx->buf) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->buf);
  }
  if (ctx->rsu_scratch) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->rsu_scratch);
  }
  delete ctx;
}

}  // extern "C"
