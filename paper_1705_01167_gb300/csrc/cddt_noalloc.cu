// cddt_noalloc.cu -- slice-sorted ray casting that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc while they run: a host application
// that reserves all device memory up front and hands libraries fixed
// budgets, or a real-time loop that forbids allocation after start-up.
// cddt_calc_range_many(..., sort_by_slice = 1, ...) grows a per-handle
// scratch with cudaMalloc; this entry point runs the same kernels on a fixed
// buffer that is part of the library's device image instead.
#include <cuda_runtime.h>

#include <mutex>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

namespace {

// Largest inputs the fixed buffer holds.
constexpr int64_t kMaxQueries = CDDT_NOALLOC_MAX_QUERIES;
constexpr int64_t kMaxBuckets = cddt::kMaxSortBuckets;
constexpr int64_t kMaxBlocks = (kMaxQueries + cddt::kSortTile - 1) / cddt::kSortTile;
constexpr int64_t kMaxCounts = kMaxBuckets * kMaxBlocks;
// scan partials and total + (bucket, block) counts + alignment + one
// 16-byte record per query (the layout of the sorted path's scratch; the
// call checks the exact size before it launches anything)
constexpr size_t kScratchBytes = 8 * (kMaxCounts / 4096 + 4) + 4 * kMaxCounts + 16 + 16 * kMaxQueries;

// The buffer itself.  Host code must not pass its name to a kernel (in host
// code it is only a stand-in for the symbol); its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_addr[kMaxDevices] = {};

cddt_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return CDDT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return CDDT_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CDDT_OK;
}

}  // namespace

extern "C" cddt_status cddt_calc_range_many_noalloc(cddt_t h, const float *pose_dev, float *range_dev, int64_t n,
                                                    void *stream)
{
    CDDT_RANGE("cddt_calc_range_many_noalloc", stream);
    if (!h) return CDDT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CDDT_ERR_CUDA;
    if (dev != h->device) return CDDT_ERR_ARG;
    if (n < 0 || n > kMaxQueries || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    if (h->N > CDDT_NOALLOC_MAX_THETA_DISC) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_calc_range_many_noalloc");
    void *scratch = nullptr;
    cddt_status rc = scratch_address(dev, &scratch);
    if (rc != CDDT_OK) return rc;
    if (n == 0) return CDDT_OK;
    if (cddt::sorted_scratch_bytes(h, n) > (int64_t)kScratchBytes) return CDDT_ERR_ARG;
    return cddt::calc_range_sorted_into(h, pose_dev, range_dev, n, scratch, (int64_t)kScratchBytes,
                                        (cudaStream_t)stream);
}
