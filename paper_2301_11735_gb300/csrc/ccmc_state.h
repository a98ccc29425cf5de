// ccmc_state.h -- launchers of the compact (2 bits a site, row-major) state
// conversions (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ccmc_internal.h"

namespace ccmc {

// in / out: N/4 bytes, site i = y Lx + x at bits 2 (i mod 4) of byte i / 4.
cudaError_t launch_pack2(const Geo &g, const uint8_t *in, cudaStream_t s);
cudaError_t launch_unpack2(const Geo &g, uint8_t *out, cudaStream_t s);

}  // namespace ccmc
