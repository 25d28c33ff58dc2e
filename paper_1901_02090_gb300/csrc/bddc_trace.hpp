// NVTX ranges over the host-side stages of setup and serving.  NVTX v3 is
// header-only: without a profiler attached the calls return at once, with
// one (ncu's --nvtx filters, Nsight) each stage shows as a named range on
// the calling thread.  The solve kernel has its own in-kernel phase
// timeline (bddc_debug_phase_times).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace bddc {

// a range from construction to destruction; next() closes it and opens the
// following stage
class TraceStage {
public:
    explicit TraceStage(const char* name) { nvtxRangePushA(name); }
    void next(const char* name) {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~TraceStage() { nvtxRangePop(); }
    TraceStage(const TraceStage&) = delete;
    TraceStage& operator=(const TraceStage&) = delete;
};

}  // namespace bddc
