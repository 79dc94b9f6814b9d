// NVTX ranges around the host entry points (initialisation, stepping,
// volumes), so that a profiler's timeline shows which library call enqueued
// which kernels.  NVTX v3 is header-only: without a profiler attached the
// push and pop are a check of a null function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace lbmk {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lbmk
