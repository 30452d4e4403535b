// kpz_internal.h -- launch interfaces between the C-ABI layer and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "kpz_common.cuh"

namespace kpz {

// Process-wide count of kernel launches issued by this library.
void count_launch(uint64_t n = 1);

// Acceptance threshold out of 2^16 for a per-attempt probability (eq. rule):
// min(65536, floor(p * 65536 + 0.5)); an attempt accepts when its uniform
// 16-bit number U < T, so p = 1 always and p = 0 never accepts.
inline uint32_t acceptance_threshold(double p) {
  if (!(p > 0.0)) return 0u;
  if (p >= 1.0) return 65536u;
  const double t = __builtin_floor(p * 65536.0 + 0.5);
  return t >= 65536.0 ? 65536u : (uint32_t)t;
}

// Bit levels of U that can still change a comparison with Tp or Tq.
inline uint32_t acceptance_levels(uint32_t Tp, uint32_t Tq) {
  const uint32_t low = (Tp & 0xFFFFu) | (Tq & 0xFFFFu);
  return low ? 16u - (uint32_t)__builtin_ctz(low) : 0u;
}

// One sweep (one MCS) of the decomposed dynamics, Sec. 3 and 3.1.
struct SweepParams {
  uint32_t* lat;            // lattice words (layout in kpz_common.cuh)
  const uint64_t* t_dev;    // device sweep counter; this launch does sweep *t_dev + s_add
  uint32_t s_add;
  Geometry g;
  uint32_t ntx, nty;        // tiles per row / per column of the tile grid
  uint32_t run;             // tiles one warp sweeps in a row per work item
  uint32_t runs_x;          // ntx / run (work items per tile row)
  uint32_t Tp, Tq;          // acceptance thresholds out of 2^16 (65536 = always)
  uint32_t nlev;            // acceptance levels that can change a decision
  uint32_t k0, k1;          // Philox key = seed
  uint32_t sample;          // realisation index (Philox counter word 3)
  unsigned long long* h00;  // absolute height of site (0,0), two's complement
  uint32_t* queue;          // single-lattice sweep: work-queue counter, 0 between launches
  uint32_t cell;            // work-group cell edge: 4 (default) or 2 (the C = 2 limit)
};

// Philox key of a seed: its low and high 32-bit words.
inline void set_philox_key(SweepParams& P, uint64_t seed) {
  P.k0 = (uint32_t)(seed & 0xffffffffu);
  P.k1 = (uint32_t)(seed >> 32);
}

cudaError_t launch_sweep(const SweepParams& P, uint32_t warps_per_cta, cudaStream_t st);
cudaError_t launch_advance(uint64_t* t_dev, uint32_t n, cudaStream_t st);
// One sweep of the tile-set variant of the device layer (kpz_tileset.cu):
// four launches, one per tile set, in the order drawn for the sweep.
cudaError_t launch_sweep_tilesets(const SweepParams& P, cudaStream_t st);
// One sweep with dead borders at both layers (kpz_db2.cu): 128 x 128 tiles.
cudaError_t launch_sweep_db2(const SweepParams& P, cudaStream_t st);
// One sweep of the random-sequential reference by colour classes (kpz_colour.cu):
// 4 * 2^m launches, one per sub-step.
cudaError_t launch_sweep_colour(const SweepParams& P, uint32_t m, cudaStream_t st);

// Observables and conversions (kpz_observe.cu).
cudaError_t launch_init_flat(uint32_t* lat, Geometry g, cudaStream_t st);
// Packed exchange format, rows [j0, j0 + nrows) <-> packed[(j - j0) * L/16 + i/16].
// The import walks the bands in order: *hcar carries the absolute height of
// site (0, j0) modulo 4 from band to band; hcol is scratch for nrows int32.
cudaError_t launch_export_packed(const uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 uint32_t* packed, cudaStream_t st);
cudaError_t launch_import_packed(uint32_t* lat, Geometry g, uint32_t j0, uint32_t nrows,
                                 const uint32_t* packed, uint32_t* hcar, int32_t* hcol,
                                 cudaStream_t st);

// Exact height sums, eq. Wdef: col0[L] (int32) and acc[3] (S1, S2 lo, S2 hi)
// are scratch that the caller provides.
cudaError_t launch_roughness(const uint32_t* lat, Geometry g, int32_t* col0,
                             unsigned long long* acc, cudaStream_t st);
// Heights of rows [j0, j0 + nrows) into out[(j - j0) * L + i], gauge h(0,0) = 0
// plus *h00 when h00 is not null; needs col0 filled by launch_col0.
cudaError_t launch_col0(const uint32_t* lat, Geometry g, int32_t* col0, cudaStream_t st);
cudaError_t launch_heights(const uint32_t* lat, Geometry g, const int32_t* col0, uint32_t j0,
                           uint32_t nrows, const unsigned long long* h00, int64_t* out,
                           cudaStream_t st);

}  // namespace kpz
