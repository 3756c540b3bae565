// trace.h -- optional NVTX ranges around the library's coarse steps (a search,
// a batched launch, a server batch), for profilers that show or filter by them
// (Nsight Systems timelines, ncu --nvtx).  Off unless the environment has
// WXPY_NVTX=1, read once; the per-call entry points carry no range at all.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace wx {

bool trace_enabled();

// Pushes a range for its lifetime when tracing is on.
class TraceRange {
  public:
    explicit TraceRange(const char *name) : on_(trace_enabled()) {
        if (on_) nvtxRangePushA(name);
    }
    ~TraceRange() {
        if (on_) nvtxRangePop();
    }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

  private:
    bool on_;
};

}  // namespace wx
