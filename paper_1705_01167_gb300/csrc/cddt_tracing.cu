// cddt_tracing.cu -- the optional CUDA-event trace of the C-ABI calls: each
// traced call records an event on its stream at entry and at exit; the pairs
// are timed when the trace is folded (on report, or when many are pending)
// and summed per entry point.  Off unless cddt_trace_enable(1) is called or
// CDDT_TRACE=1 is set; when off a call pays one atomic load.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cddt_trace.cuh"

namespace cddt {
namespace {

struct Pending {
    const char *name;
    cudaEvent_t a, b;
};
struct Agg {
    int64_t calls = 0;
    double total = 0, lo = 0, hi = 0;  // milliseconds
};

std::atomic<int> g_on{-1};  // -1: CDDT_TRACE not read yet
std::mutex g_mu;
std::vector<Pending> g_pending;
std::map<std::string, Agg> g_agg;
constexpr size_t kMaxPending = 1 << 14;  // fold (and free the events) beyond this

// Time and release every pending pair; caller holds g_mu.
void fold_locked()
{
    for (const Pending &p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Agg &g = g_agg[p.name];
            g.lo = g.calls ? std::min(g.lo, (double)ms) : (double)ms;
            g.hi = g.calls ? std::max(g.hi, (double)ms) : (double)ms;
            g.total += ms;
            ++g.calls;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
    cudaGetLastError();  // a failed sync above must not leak into the next call's status
}

}  // namespace

bool trace_on()
{
    int v = g_on.load(std::memory_order_relaxed);
    if (v < 0) {
        const char *e = std::getenv("CDDT_TRACE");
        v = (e && !std::strcmp(e, "1")) ? 1 : 0;
        int expected = -1;
        g_on.compare_exchange_strong(expected, v);
        v = g_on.load(std::memory_order_relaxed);
    }
    return v == 1;
}

void trace_begin(cudaStream_t st, cudaEvent_t &a)
{
    a = nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    if (cudaEventCreate(&a) != cudaSuccess) {
        cudaGetLastError();
        a = nullptr;
        return;
    }
    if (cudaEventRecord(a, st) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(a);
        a = nullptr;
    }
}

void trace_end(const char *name, cudaStream_t st, cudaEvent_t a)
{
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess) {
        cudaGetLastError();
        if (b) cudaEventDestroy(b);
        cudaEventDestroy(a);
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({name, a, b});
    if (g_pending.size() >= kMaxPending) fold_locked();
}

}  // namespace cddt

extern "C" {

cddt_status cddt_trace_enable(int32_t on)
{
    if (on != 0 && on != 1) return CDDT_ERR_ARG;
    cddt::g_on.store(on, std::memory_order_relaxed);
    return CDDT_OK;
}

cddt_status cddt_trace_report(char *buf, int64_t cap, int64_t *len)
{
    if (cap < 0 || (cap > 0 && !buf)) return CDDT_ERR_ARG;
    std::string out = "entry,calls,total_ms,mean_ms,min_ms,max_ms\n";
    {
        std::lock_guard<std::mutex> lk(cddt::g_mu);
        cddt::fold_locked();
        char line[256];
        for (const auto &kv : cddt::g_agg) {
            const cddt::Agg &g = kv.second;
            std::snprintf(line, sizeof(line), "%s,%lld,%.6f,%.6f,%.6f,%.6f\n", kv.first.c_str(),
                          (long long)g.calls, g.total, g.total / (double)g.calls, g.lo, g.hi);
            out += line;
        }
        cddt::g_agg.clear();
    }
    if (len) *len = (int64_t)out.size() + 1;
    if (cap > 0) {
        const size_t n = std::min<size_t>(out.size(), (size_t)cap - 1);
        std::memcpy(buf, out.data(), n);
        buf[n] = '\0';
    }
    return CDDT_OK;
}

}  // extern "C"
