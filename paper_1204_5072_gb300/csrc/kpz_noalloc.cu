// kpz_noalloc.cu -- exact W^2 of a device-resident lattice with no allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// width: processes whose device memory is fully reserved by another
// framework's caching allocator, or real-time loops that must not allocate
// after start-up.
// kpz_roughness_static gives them the reduction of kpz_roughness on a lattice
// they already hold (the pointer kpz_device_lattice returns), with its scratch
// (column-0 heights and three 64-bit accumulators) in the file-scope array
// below instead of memory the library would allocate.
#include <mutex>

#include "kpz.h"
#include "kpz_internal.h"

using namespace kpz;

namespace {

constexpr uint32_t kMaxL = 131072;  // largest lattice the static scratch serves
constexpr size_t kAccOffset = (size_t)kMaxL * sizeof(int32_t);  // 256-byte aligned
// Column-0 heights (kMaxL int32) followed by the three accumulators:
// 512 KiB + 256 B, held by every GPU that loads the library until exit.
static __device__ __align__(256) int32_t g_scratch[kMaxL + 64];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

bool valid_size(uint32_t L) { return L >= 128u && (L & (L - 1u)) == 0u; }

}  // namespace

extern "C" kpz_status kpz_roughness_static(const void* lattice_dev, uint32_t L, uint32_t parity,
                                           void* stream, kpz_rough* out) {
  if (!lattice_dev || !out || !valid_size(L)) return KPZ_EINVAL;
  if (L > kMaxL) return KPZ_ERANGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KPZ_ENODEV;
  void* base = nullptr;
  {
    // First call on this device (which is current): look up the device
    // address of the static array once and remember it for the process (a
    // device reset invalidates it; the header says so).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return KPZ_ECUDA;
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  int32_t* col0 = static_cast<int32_t*>(base);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + kAccOffset);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Geometry g{};
  g.L = L;
  g.NR = L / 4;
  g.NB = L / 128;
  g.par = parity & 1u;
  // launch_roughness zeroes the accumulators before it adds into them.
  if (launch_roughness(static_cast<const uint32_t*>(lattice_dev), g, col0, acc, st) != cudaSuccess)
    return KPZ_ECUDA;
  unsigned long long host[3];
  if (cudaMemcpyAsync(host, acc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return KPZ_ECUDA;
  const uint64_t N = (uint64_t)L * L;
  out->t_mcs = 0;
  out->n_sites = N;
  out->sum_h = (int64_t)host[0];
  out->sum_h2_lo = host[1];
  out->sum_h2_hi = host[2];
  out->h00 = 0;
  const unsigned __int128 S2 = ((unsigned __int128)host[2] << 64) | host[1];
  const __int128 S1 = (int64_t)host[0];
  const unsigned __int128 num = (unsigned __int128)N * S2 - (unsigned __int128)(S1 * S1);
  out->w2 = (double)num / ((double)N * (double)N);
  return KPZ_OK;
}
