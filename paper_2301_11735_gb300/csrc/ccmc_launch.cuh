// ccmc_launch.cuh -- host-side launch helpers shared by the kernel files.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ccmc {

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel of the stream drains, and waits for it (griddepcontrol)
// before touching anything that kernel writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, int block, size_t smem,
                                   cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, int block, cudaStream_t s,
                              Args... args) {
  return launch_pdl_smem(kernel, grid, block, 0, s, args...);
}

inline int grid_for(int64_t items, int block, int cap) {
  int64_t b = (items + block - 1) / block;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace ccmc
