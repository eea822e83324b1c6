// NVTX ranges around the library's step and training calls, so that a
// profiler (ncu --nvtx, nsys) can attribute kernels to the API call that
// queued them.  NVTX v3 is header-only: without a profiler attached the push
// and pop are no-ops.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace trace {

struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace trace
