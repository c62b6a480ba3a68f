// cddt_lut.cu -- the three-dimensional lookup table the paper compares the
// CDDT against (Section II; 16-bit entries, Table I): a range for every
// discrete state (cell centre, theta_k), built on the GPU by casting every
// state through a CDDT, and read by a ray cast and a fused sensor model that
// snap each query to its state.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

struct cddt_lut_s {
    int device = 0;
    int32_t W = 0, H = 0, N = 0;
    float max_range = 0, scale = 1, inv_scale = 1, inv_step = 0;
    uint16_t *table = nullptr;  // [N][H][W]
};

namespace cddt {

// The 16-bit code of a range (reading L1): r * scale rounded half up, scale a
// power of two (exact products), at most 65535.
__device__ __forceinline__ uint16_t lut_code(float r, float scale)
{
    const float w = floorf(__fadd_rn(__fmul_rn(r, scale), 0.5f));
    return (uint16_t)fminf(fmaxf(w, 0.0f), 65535.0f);
}

// Every state of one theta_k per block row: the cast from the cell centre
// (i, j) in direction theta[k] = 2 pi k / N (computed in double on the host,
// stored float32).
template <typename KT, int SEARCH>
__global__ void lut_build_kernel(MapView m, const float *theta, uint16_t *table, float scale)
{
    const uint64_t pol = policy_evict_last();
    const int64_t cells = (int64_t)m.W * m.H;
    const int64_t total = cells * m.N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / cells);
        const int64_t q = t - (int64_t)k * cells;
        const int j = (int)(q / m.W), i = (int)(q - (int64_t)j * m.W);
        const float th = __ldg(theta + k);
        Cast c;
        c.r = 0.0f;
        if (free_cell(m.grid, m.W, m.H, (float)i, (float)j)) {
            int kk;
            if (query_dir(th, m.inv_step, m.N, kk)) {
                Cast f, b;
                bool kf;
                cast_pair<KT, SEARCH>(m, (float)i, (float)j, kk, false, pol, f, b, kf);
                c = kf ? f : b;
            }
        }
        table[t] = lut_code(c.r, scale);
    }
}

// The state of a query: nearest cell centre (off the map: none) and its
// direction index; the table's range there.
__device__ __forceinline__ float lut_range(const uint16_t *table, int W, int H, int N, float inv_step,
                                           float inv_scale, float x, float y, float th)
{
    const float fx = floorf(__fadd_rn(x, 0.5f)), fy = floorf(__fadd_rn(y, 0.5f));
    if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) return 0.0f;
    int k;
    if (!query_dir(th, inv_step, N, k)) return 0.0f;
    const uint16_t code = __ldg(table + ((int64_t)k * H + (int)fy) * W + (int)fx);
    return __fmul_rn((float)code, inv_scale);
}

__global__ void lut_calc_range_kernel(cddt_lut_s L, const float *pose, float *out, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = lut_range(L.table, L.W, L.H, L.N, L.inv_step, L.inv_scale, __ldg(pose + 3 * q),
                           __ldg(pose + 3 * q + 1), __ldg(pose + 3 * q + 2));
}

// The fused sensor model over the table: one thread per particle, every
// beam a table read (no search, no pairing); filters are segments of the
// particle array, each with its own scan obs [F][B].
__global__ void lut_sensor_kernel(cddt_lut_s L, const float *part, int64_t P, const int64_t *seg, int F,
                                  const float *beam_off, const float *obs, int B, BeamConsts bc, float *logw)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = F - 1;  // the particle's filter
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(seg + mid) <= p) lo = mid;
            else hi = mid - 1;
        }
        const float *ob = obs + (int64_t)lo * B;
        const float x = __ldg(part + 3 * p), y = __ldg(part + 3 * p + 1), th = __ldg(part + 3 * p + 2);
        float acc = 0.0f, dl;
        for (int i = 0; i < B; ++i) {
            const float r = lut_range(L.table, L.W, L.H, L.N, L.inv_step, L.inv_scale, x, y,
                                      __fadd_rn(th, __ldg(beam_off + i)));
            const BeamObs o = beam_obs(bc, __ldg(ob + i));
            acc += beam_log2p<false>(bc, o, r, dl);
        }
        logw[p] = acc * kLn2;
    }
}

}  // namespace cddt

extern "C" {

cddt_status cddt_lut_build(cddt_t h, void *stream, cddt_lut *out)
{
    CDDT_RANGE("cddt_lut_build", stream);
    if (!h || !out) return CDDT_ERR_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_lut_build");
    const int64_t n = (int64_t)h->W * h->H * h->N;
    cddt_lut_s *L = new cddt_lut_s();
    L->device = h->device;
    L->W = h->W;
    L->H = h->H;
    L->N = h->N;
    L->max_range = h->max_range;
    int e;
    std::frexp(65535.0 / (double)h->max_range, &e);  // 2^(e-1) <= 65535 / max_range < 2^e
    L->scale = (float)std::ldexp(1.0, e - 1);
    L->inv_scale = (float)std::ldexp(1.0, 1 - e);
    L->inv_step = (float)((double)h->N / (2.0 * 3.14159265358979323846));
    if (cudaMalloc(&L->table, sizeof(uint16_t) * (size_t)n) != cudaSuccess) {
        delete L;
        return CDDT_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the N table directions, one float each (the kernel reads them instead
    // of evaluating the double expression per state)
    std::vector<float> th_h((size_t)h->N);
    for (int k = 0; k < h->N; ++k) th_h[k] = (float)((2.0 * 3.14159265358979323846 * (double)k) / (double)h->N);
    float *th = nullptr;
    if (cudaMallocAsync(&th, sizeof(float) * th_h.size(), st) != cudaSuccess) {
        cudaFree(L->table);
        delete L;
        return CDDT_ERR_OOM;
    }
    // the pageable source is consumed before the call returns
    cudaError_t ce = cudaMemcpyAsync(th, th_h.data(), sizeof(float) * th_h.size(), cudaMemcpyHostToDevice, st);
    const cddt::MapView m = h->view();
    const unsigned blocks = cddt::grid_cap(n, 256, 64);
    const bool bin = h->search == CDDT_SEARCH_BINARY;
    if (ce == cudaSuccess) {
        if (h->u16 && bin)
            cddt::lut_build_kernel<uint16_t, CDDT_SEARCH_BINARY><<<blocks, 256, 0, st>>>(m, th, L->table, L->scale);
        else if (h->u16)
            cddt::lut_build_kernel<uint16_t, CDDT_SEARCH_TREE><<<blocks, 256, 0, st>>>(m, th, L->table, L->scale);
        else if (bin)
            cddt::lut_build_kernel<float, CDDT_SEARCH_BINARY><<<blocks, 256, 0, st>>>(m, th, L->table, L->scale);
        else
            cddt::lut_build_kernel<float, CDDT_SEARCH_TREE><<<blocks, 256, 0, st>>>(m, th, L->table, L->scale);
        ce = cudaGetLastError();
    }
    cudaFreeAsync(th, st);
    if (ce != cudaSuccess) {
        cudaFree(L->table);
        delete L;
        return CDDT_ERR_CUDA;
    }
    *out = L;
    return CDDT_OK;
}

cddt_status cddt_lut_destroy(cddt_lut L)
{
    if (!L) return CDDT_OK;
    cudaDeviceSynchronize();
    cudaFree(L->table);
    delete L;
    return CDDT_OK;
}

cddt_status cddt_lut_info(cddt_lut L, int64_t *bytes, float *scale)
{
    if (!L) return CDDT_ERR_ARG;
    if (bytes) *bytes = (int64_t)sizeof(uint16_t) * L->W * L->H * L->N;
    if (scale) *scale = L->scale;
    return CDDT_OK;
}

cddt_status cddt_lut_calc_range_many(cddt_lut L, const float *pose_dev, float *range_dev, int64_t n, void *stream)
{
    CDDT_RANGE("cddt_lut_calc_range_many", stream);
    if (!L || n < 0 || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_lut_calc_range_many");
    if (n == 0) return CDDT_OK;
    cddt::lut_calc_range_kernel<<<cddt::grid_cap(n, 256, 64), 256, 0, (cudaStream_t)stream>>>(*L, pose_dev,
                                                                                                   range_dev, n);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

cddt_status cddt_lut_sensor_weights(cddt_lut L, const float *particles_dev, int64_t P, const int64_t *seg_start_dev,
                                    int32_t F, const float *beam_off_dev, const float *obs_dev, int32_t B,
                                    const cddt_beam_model *m, float *logw_dev, void *stream)
{
    CDDT_RANGE("cddt_lut_sensor_weights", stream);
    if (!L || P < 0 || F < 1 || B < 1 || !m) return CDDT_ERR_ARG;
    if (P > 0 && (!particles_dev || !seg_start_dev || !beam_off_dev || !obs_dev || !logw_dev)) return CDDT_ERR_ARG;
    if (!(m->sigma_hit > 0) || !(m->max_range > 0) || !(m->lambda_short > 0)) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_lut_sensor_weights");
    if (P == 0) return CDDT_OK;
    cddt::lut_sensor_kernel<<<cddt::grid_cap(P, 256, 64), 256, 0, (cudaStream_t)stream>>>(
        *L, particles_dev, P, seg_start_dev, F, beam_off_dev, obs_dev, B, cddt::make_beam_consts(*m), logw_dev);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

}  // extern "C"
