// ccmc_fault.h -- host-side fault injection for testing the library's failure
// paths without faulting a GPU.  The environment variable CCMC_FAULT, read at
// each call, holds comma-separated fault names:
//   alloc  : handle creation fails as if device memory ran out (CCMC_E_NOMEM),
//            before anything is allocated or any CUDA call is made;
//   launch : sweep calls fail as if a kernel launch failed (CCMC_E_CUDA),
//            before anything is queued, leaving the handle usable;
//   admit  : the server refuses every request at admission as if it could
//            never fit the memory budget (result status CCMC_E_BUDGET).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

namespace ccmc {

// One CTA waits, at most `polls` polls, on an mbarrier nothing completes and
// sets *status to 1 when it gives up (ccmc_kernels.cu).
cudaError_t launch_wait_selftest(uint32_t polls, int *status, cudaStream_t s);

inline bool fault_injected(const char *what) {
  const char *v = std::getenv("CCMC_FAULT");
  if (!v || !*v) return false;
  const size_t n = std::strlen(what);
  for (const char *p = v; *p;) {
    const char *e = std::strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : std::strlen(p);
    if (len == n && std::strncmp(p, what, n) == 0) return true;
    if (!e) break;
    p = e + 1;
  }
  return false;
}

}  // namespace ccmc
