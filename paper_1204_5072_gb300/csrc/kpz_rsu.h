// kpz_rsu.h -- launch interface of the exact random-sequential sweep (kpz_rsu.cu).
#pragma once
#include "kpz_internal.h"

namespace kpz {

// Device bytes of scratch one sweep of an L x L lattice needs (per-site attempt
// buckets and progress counters, about 20 L^2 bytes).
size_t rsu_scratch_bytes(uint32_t L);
// One sweep of random-sequential updates equal bit for bit to making the L^2
// attempts one at a time; `scratch` holds rsu_scratch_bytes(L) device bytes.
// Synchronises st (the host polls the number of attempts made).
cudaError_t launch_sweep_rsu(const SweepParams& P, void* scratch, cudaStream_t st);

}  // namespace kpz
