// cddt_kernels.cuh -- host-side entry points shared between the translation
// units of libcddt.so (scan, layout, sort/index, construction).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cddt_internal.cuh"

namespace cddt {

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *scratch,
                        uint64_t *total_dev, cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);
cddt_status layout_bins(cddt_s *h, uint32_t *count_dev, cudaStream_t st, void **store_out,
                        int64_t *nodes_out, int64_t extra_nodes);
cddt_status sort_and_index_any(cddt_s *h, cudaStream_t st);
cddt_status construct(cddt_s *h, cudaStream_t st);
cddt_status init_handle(cddt_s *h, const uint8_t *grid_dev, cudaStream_t st);
cddt_status prune(cddt_s *h, cudaStream_t st);
cddt_status update_cells(cddt_s *h, const int32_t *xy, const uint8_t *occ, int32_t n,
                         cudaStream_t st);

// Arguments of the sensor-model kernels (cddt_query.cu).
struct SensorArgs {
    const float *part;
    int64_t P;
    const float *beam_off;
    const float *obs;
    int32_t B, D;
    BeamConsts bc;
    float *logw;
    float *ranges;
    const float *grad_logw;
    float *grad_xy;
    unsigned long long *work;  // work-count mode: 6 counters
};
cddt_status launch_sensor(const cddt_s *h, const SensorArgs &a, int mode, cudaStream_t st);
cddt_status calc_range(cddt_s *h, const float *pose, float *out, int64_t n, int sorted, cudaStream_t st);
// The slice-sorted cast on caller-provided scratch of sorted_scratch_bytes(h, n)
// bytes (cddt_query.cu); returns CDDT_ERR_ARG when the scratch is too small.
int64_t sorted_scratch_bytes(const cddt_s *h, int64_t n);
cddt_status calc_range_sorted_into(cddt_s *h, const float *pose, float *out, int64_t n, void *scratch,
                                   int64_t scratch_bytes, cudaStream_t st);

// A device buffer freed on scope exit.
struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
    template <typename T> T *as() { return reinterpret_cast<T *>(p); }
};

template <typename KT> __device__ __forceinline__ KT pad_key();
template <> __device__ __forceinline__ float pad_key<float>() { return kInf; }
template <> __device__ __forceinline__ uint16_t pad_key<uint16_t>() { return 0xffffu; }

// First key of a bin's leaf run.
template <typename KT>
__device__ __forceinline__ KT *leaf_run(void *store, uint32_t off, uint32_t n)
{
    constexpr int LK = KeyT<KT>::LK;
    return reinterpret_cast<KT *>(store) + ((size_t)(off + internal_nodes(n, LK, KeyT<KT>::R)) << LK);
}

// The segments of a segmented sort: the leaf runs of a store's bins (hdr
// set), or plain ranges base[off[id] .. off[id] + len[id]).
template <typename KT>
struct Segs {
    void *store;
    const BinHdr *hdr;
    KT *base;
    const uint32_t *off;
    const uint32_t *len;
    __device__ __forceinline__ void get(uint32_t id, KT *&p, uint32_t &n) const
    {
        if (hdr) {
            n = bin_count(hdr[id].nm);
            p = leaf_run<KT>(store, hdr[id].off, n);
        } else {
            n = len[id];
            p = base + off[id];
        }
    }
};

// Sort every segment ascending (cddt_build.cu).  Synchronises `st`.
template <typename KT>
cddt_status sort_segments(const Segs<KT> &sg, int64_t nseg, cudaStream_t st);
// Fill the trees and headers of every bin from the sorted leaf runs.
cddt_status index_store(cddt_s *h, cudaStream_t st);
// Slice tables' eps for pruning: 32 units in the last place of the largest
// projected coordinate.
float prune_eps(int W, int H);

inline unsigned grid_cap(int64_t n, int threads, int64_t cap = 152 * 64)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace cddt
