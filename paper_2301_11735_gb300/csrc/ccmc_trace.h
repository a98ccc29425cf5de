// ccmc_trace.h -- host-side trace ranges (NVTX, header-only): a profiler or
// tracer attached to the process shows the library's calls and the server's
// slices as named ranges; without one, each range costs two no-op calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ccmc {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace ccmc
