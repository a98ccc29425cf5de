// ccmc_map.h -- the paper-faithful map mode's device launcher (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ccmc_internal.h"

namespace ccmc {

// One map (Sec. 3.2): npairs non-interacting pairs, site indices y * Lx + x of
// a then b in d_pairs (device memory), map index m keying the random words.
cudaError_t launch_map(const Geo &g, const int32_t *d_pairs, int64_t npairs, uint64_t m,
                       const DevTables &t, cudaStream_t s);

}  // namespace ccmc
