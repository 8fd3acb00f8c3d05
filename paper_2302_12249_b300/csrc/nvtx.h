// nvtx.h -- NVTX ranges (domain "merf") around the library's host-side phases, for Nsight
// timelines and for selecting kernels in ncu (--nvtx --nvtx-include "merf@merf_render/"): scene
// upload, render and trace launches, the host-output renders, the adjoint, and each serving
// iteration's launch and image copy.  NVTX v3 is header-only; with no tool attached a range
// costs a call through an empty function pointer.  The deferred MLP runs inside the render
// kernels (after compositing, in the same thread), so it has no host-side range of its own.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace merf {

inline nvtxDomainHandle_t nvtx_domain()
{
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("merf");
    return d;
}

class NvtxRange {
public:
    explicit NvtxRange(const char *name)
    {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace merf
