// fd_trace.h -- NVTX ranges over the C ABI's calls, for Nsight tools.
//
// Host code only.  With no tool attached, a range costs one call into the NVTX
// stub (no allocation, no synchronisation).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace fdk {

// Marks the lifetime of one API call as a named range.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace fdk
