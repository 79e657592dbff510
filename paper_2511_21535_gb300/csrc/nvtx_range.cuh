// Named ranges on the host timeline for profilers (NVTX, header-only: each
// call is a no-op unless a profiling tool is attached to the process).  Every
// C entry point that queues device work opens one for its duration, so a
// timeline shows the paper's phases (tree build, restructuring, operator,
// host copies) around the kernels they launch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace p2p {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace p2p
