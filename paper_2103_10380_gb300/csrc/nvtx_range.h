// nvtx_range.h -- named NVTX ranges around the library's host entry points and
// served batches, for timeline tools (Nsight Systems, ncu's NVTX filters). The
// NVTX v3 headers are header-only: without an attached tool a range costs a
// branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace fnr {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace fnr
