// NVTX ranges around the library's entry points, so that a profiler's
// timeline (ncu --nvtx, Nsight Systems) shows which call a kernel belongs
// to.  NVTX v3 is header-only: without a tool attached each range is a
// cheap no-op.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sbg {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace sbg
