// Tracing of the host entry points: an NVTX range per call, visible to Nsight Systems and to
// `ncu --nvtx`; NVTX is header-only and its calls are no-ops when no tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace lbm
