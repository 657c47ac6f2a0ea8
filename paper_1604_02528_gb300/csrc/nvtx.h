// NVTX ranges (header-only NVTX 3: without an attached tool every call is a
// check of a function pointer).  Every public entry point opens a range named
// after itself; a schedule issued kernel by kernel (or captured into its CUDA
// graph) opens one per tree level and launch kind, "L<level> <kind>".
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdio>

namespace selinv {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// name of a launch kind (KL_*) for the ranges
const char *launch_kind_name(int kind);

}  // namespace selinv
