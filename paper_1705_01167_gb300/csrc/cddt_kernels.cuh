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

inline unsigned grid_cap(int64_t n, int threads, int64_t cap = 152 * 64)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace cddt
