// cddt_trace.cuh -- NVTX ranges around the C-ABI calls (shown by Nsight
// tools, no-ops without one attached), an optional CUDA-event trace of the
// same calls (cddt_trace_enable / cddt_trace_report, or CDDT_TRACE=1), and
// the host-side fault injection read from the CDDT_FAULT environment
// variable.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>
#include <cstring>

#include "../../include/cddt.h"

namespace cddt {

// Event trace (implemented in cddt_api.cu): when on, each call records a
// CUDA event on its stream at entry and at exit (not while the stream is
// being captured into a graph); the pairs are timed and summed per entry
// point when the trace is reported.
bool trace_on();
void trace_begin(cudaStream_t st, cudaEvent_t &a);
void trace_end(const char *name, cudaStream_t st, cudaEvent_t a);

struct Range {
    Range(const char *name, void *stream) : name_(name), st_(static_cast<cudaStream_t>(stream))
    {
        nvtxRangePushA(name);
        if (trace_on()) trace_begin(st_, a_);
    }
    ~Range()
    {
        if (a_) trace_end(name_, st_, a_);
        nvtxRangePop();
    }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;

  private:
    const char *name_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr;
};

// CDDT_FAULT=<kind>[:<entry point>] makes the named C-ABI entry point (every
// entry point with a fault point when no name is given) return the status of
// that failure after its argument checks and before it touches the device:
// oom -> CDDT_ERR_OOM (a device allocation failed), launch -> CDDT_ERR_CUDA
// (a launch or copy failed), timeout -> CDDT_ERR_TIMEOUT (a bounded wait gave
// up).  The handle or plan is left as it was.  Any other value injects
// nothing.  Read on every call, so a test can set and clear it.
inline cddt_status injected_fault(const char *entry)
{
    const char *v = std::getenv("CDDT_FAULT");
    if (!v || !*v) return CDDT_OK;
    const char *colon = std::strchr(v, ':');
    const size_t kl = colon ? (size_t)(colon - v) : std::strlen(v);
    if (colon && std::strcmp(colon + 1, entry) != 0) return CDDT_OK;
    if (kl == 3 && !std::strncmp(v, "oom", 3)) return CDDT_ERR_OOM;
    if (kl == 6 && !std::strncmp(v, "launch", 6)) return CDDT_ERR_CUDA;
    if (kl == 7 && !std::strncmp(v, "timeout", 7)) return CDDT_ERR_TIMEOUT;
    return CDDT_OK;
}

}  // namespace cddt

#define CDDT_RANGE(name, stream) cddt::Range cddt_range_(name, stream)
#define CDDT_FAULT_POINT(name)                                                \
    do {                                                                      \
        cddt_status f_ = cddt::injected_fault(name);                          \
        if (f_ != CDDT_OK) return f_;                                         \
    } while (0)
