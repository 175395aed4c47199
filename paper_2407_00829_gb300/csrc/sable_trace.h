// NVTX ranges around the library's phases (extract, upload, autotune, the
// device inspector, each SpMV / SpMM / batch call), so that a profiler can
// attribute time and filter kernels by phase.  The NVTX v3 header is
// header-only: without a tool attached each range costs a check of an
// uninitialised function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sable {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace sable
