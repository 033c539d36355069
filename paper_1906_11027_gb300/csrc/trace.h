// trace.h -- NVTX ranges over calls of the C ABI, so that a timeline profiler
// shows the library's calls around their kernels.  NVTX 3 is header-only and
// costs nothing when no profiler is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lbm
