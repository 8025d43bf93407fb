// trace.h -- NVTX ranges around the library's host entry points, in the domain "sird_pso", so
// that a timeline profiler shows calibrate / polish / batch runs with the kernels they launch.
// NVTX v3 is header-only: with no profiler attached a range costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sird {

inline nvtxDomainHandle_t trace_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("sird_pso");
    return d;
}

// Pushes a named range on construction and pops it on destruction (every return path).
class TraceRange {
public:
    explicit TraceRange(const char* name) {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace sird
