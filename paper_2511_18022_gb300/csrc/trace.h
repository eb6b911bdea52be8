// Internal: NVTX ranges around the C ABI's entry points (header-only NVTX 3:
// without a profiler attached a range costs one check of a function pointer).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace cvrpsd {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace cvrpsd

#define CVRPSD_TRACE(name) ::cvrpsd::TraceRange cvrpsd_trace_range_(name)
