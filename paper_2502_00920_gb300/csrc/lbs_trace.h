// Tracing of liblbs's host calls: NVTX ranges that name them in profiler
// timelines (ncu --nvtx, nsys); free when no tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace lbs {

// an NVTX range over the lifetime of the object
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace lbs
