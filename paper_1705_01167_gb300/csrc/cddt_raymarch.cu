// cddt_raymarch.cu -- the ray marching caster (Section II, the paper's "RM"
// baseline): a precomputed Euclidean distance transform of the occupancy
// grid, and a march that advances each ray by the transform's value at the
// cell it stands on until that cell is occupied.  A second baseline family
// beside the CDDT and the Bresenham walk, one thread per ray.
//
// The transform is exact and integer until the last step: a column sweep
// gives every cell's vertical distance g to the nearest occupied cell of its
// column, then each row takes the lower envelope of the parabolas
// (i - k)^2 + g_k^2 over its columns k (the separable form of the squared
// Euclidean distance), built in shared memory by one thread and read by all.
#include <cuda_runtime.h>

#include <cmath>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

struct cddt_rm_s {
    int device = 0;
    int32_t W = 0, H = 0;
    float max_range = 0;
    float *dist = nullptr;  // [H][W] distance to the nearest occupied cell centre
};

namespace cddt {

constexpr uint16_t kNoObstacle = 0xFFFF;  // column without an occupied cell

// Column sweep: g(i, j) = min |j - j'| over occupied (i, j') of column i, or
// kNoObstacle.  One thread per column; a warp's loads and stores of one row
// are 32 consecutive cells.
__global__ void edt_columns_kernel(const uint8_t *grid, int W, int H, uint16_t *g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W) return;
    uint32_t d = kNoObstacle;
    for (int j = 0; j < H; ++j) {
        const int64_t c = (int64_t)j * W + i;
        d = __ldg(grid + c) ? 0u : (d == kNoObstacle ? d : d + 1u);
        g[c] = (uint16_t)d;
    }
    d = kNoObstacle;
    for (int j = H - 1; j >= 0; --j) {
        const int64_t c = (int64_t)j * W + i;
        d = __ldg(grid + c) ? 0u : (d == kNoObstacle ? d : d + 1u);
        if (d < g[c]) g[c] = (uint16_t)d;
    }
}

// Row pass, one block per row j.  Parabola k (a column with g_k finite) is
// f_k(i) = (i - k)^2 + g_k^2; the squared distance of cell (i, j) is the
// least f_k(i).  Thread 0 keeps the lower envelope as a stack of parabolas
// v[q] with the first cell z[q] where each is least: parabola k takes over
// from an earlier k' at the smallest integer i with f_k(i) <= f_k'(i),
// ceil(((k^2 + g_k^2) - (k'^2 + g_k'^2)) / (2 (k - k'))), in 64-bit integers.
// Every thread then finds its cells' parabolas by binary search over z.  A
// map without an occupied cell gets W + H everywhere.
__global__ void edt_rows_kernel(const uint16_t *g, int W, int H, float *dist)
{
    extern __shared__ uint16_t sm[];
    uint16_t *gs = sm, *v = sm + W, *z = sm + 2 * W;
    __shared__ int m_s;
    const int j = blockIdx.x;
    const uint16_t *grow = g + (int64_t)j * W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) gs[i] = grow[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;  // stack size
        for (int k = 0; k < W; ++k) {
            const int64_t gk = gs[k];
            if (gk == kNoObstacle) continue;
            const int64_t fk = (int64_t)k * k + gk * gk;
            int64_t b = 0;
            while (m > 0) {
                const int64_t kp = v[m - 1], gp = gs[kp];
                const int64_t num = fk - (kp * kp + gp * gp), den = 2 * ((int64_t)k - kp);
                b = num >= 0 ? (num + den - 1) / den : -((-num) / den);  // ceil(num / den), den > 0
                if (b <= (int64_t)z[m - 1]) --m;
                else break;
            }
            if (m == 0) b = 0;
            if (b >= W) continue;  // never least inside the row
            v[m] = (uint16_t)k;
            z[m] = (uint16_t)b;
            ++m;
        }
        m_s = m;
    }
    __syncthreads();
    const int m = m_s;
    float *drow = dist + (int64_t)j * W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        if (m == 0) {
            drow[i] = (float)(W + H);
            continue;
        }
        int lo = 0, hi = m - 1;  // last q with z[q] <= i (z[0] = 0)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int)z[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int64_t k = v[lo], gk = gs[k], dx = (int64_t)i - k;
        drow[i] = __double2float_rn(__dsqrt_rn((double)(dx * dx + gk * gk)));
    }
}

// The march of one ray (reading RM1): c, s = dir_sincos(theta); t = 0; at
// each sample p = (fma(t, c, x), fma(t, s, y)) the cell floor(p + 1/2) is
// read: off the map ends the ray at max_range, a
// zero distance (occupied) returns t, otherwise t += distance, and t
// reaching max_range returns max_range.  A query from an occupied or off-map
// cell or with a non-finite coordinate returns 0.  steps (optional) counts
// the transform reads of each ray.  Every advance is at least 1 (a free
// cell is at least one cell from an occupied one), so a ray leaves the map
// within W + H reads; the loop bound is never reached.
__global__ void rm_kernel(const float *dist, int W, int H, const float *pose, float *out, int32_t *steps,
                          int64_t n, float max_range)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        float res = 0.0f;
        int reads = 0;
        const float fx0 = floorf(__fadd_rn(x, 0.5f)), fy0 = floorf(__fadd_rn(y, 0.5f));
        if (isfinite(x) && isfinite(y) && isfinite(th) && fx0 >= 0.0f && fx0 < (float)W && fy0 >= 0.0f &&
            fy0 < (float)H) {
            float s, c;
            dir_sincos(th, s, c);
            float t = 0.0f;
            res = max_range;
            const int kmax = W + H + 2;
            while (reads < kmax) {
                const float fx = floorf(__fadd_rn(__fmaf_rn(t, c, x), 0.5f));
                const float fy = floorf(__fadd_rn(__fmaf_rn(t, s, y), 0.5f));
                if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) break;
                const float d = __ldg(dist + (int64_t)fy * W + (int64_t)fx);
                ++reads;
                if (d == 0.0f) {
                    res = t;
                    break;
                }
                t = __fadd_rn(t, d);
                if (!(t < max_range)) break;
            }
        }
        out[q] = res;
        if (steps) steps[q] = reads;
    }
}

}  // namespace cddt

extern "C" {

cddt_status cddt_rm_build(cddt_t h, void *stream, cddt_rm *out)
{
    CDDT_RANGE("cddt_rm_build", stream);
    if (!h || !out) return CDDT_ERR_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_rm_build");
    const int W = h->W, H = h->H;
    const size_t cells = (size_t)W * H;
    const size_t smem = 3 * sizeof(uint16_t) * (size_t)W;  // g row, v, z
    if (cudaFuncSetAttribute(cddt::edt_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return CDDT_ERR_CUDA;
    cddt_rm_s *R = new cddt_rm_s();
    R->device = h->device;
    R->W = W;
    R->H = H;
    R->max_range = h->max_range;
    uint16_t *g = nullptr;
    if (cudaMalloc(&R->dist, sizeof(float) * cells) != cudaSuccess ||
        cudaMallocAsync(&g, sizeof(uint16_t) * cells, (cudaStream_t)stream) != cudaSuccess) {
        cudaFree(R->dist);
        delete R;
        return CDDT_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cddt::edt_columns_kernel<<<(W + 127) / 128, 128, 0, st>>>(h->grid, W, H, g);
    cddt::edt_rows_kernel<<<H, 256, smem, st>>>(g, W, H, R->dist);
    const cudaError_t le = cudaGetLastError();
    cudaFreeAsync(g, st);
    if (le != cudaSuccess) {
        cudaFree(R->dist);
        delete R;
        return CDDT_ERR_CUDA;
    }
    *out = R;
    return CDDT_OK;
}

cddt_status cddt_rm_destroy(cddt_rm R)
{
    if (!R) return CDDT_OK;
    cudaDeviceSynchronize();
    cudaFree(R->dist);
    delete R;
    return CDDT_OK;
}

cddt_status cddt_rm_distances(cddt_rm R, const float **dist_dev, int64_t *bytes)
{
    if (!R) return CDDT_ERR_ARG;
    if (dist_dev) *dist_dev = R->dist;
    if (bytes) *bytes = (int64_t)sizeof(float) * R->W * R->H;
    return CDDT_OK;
}

cddt_status cddt_rm_calc_range_many(cddt_rm R, const float *pose_dev, float *range_dev, int32_t *steps_dev,
                                    int64_t n, void *stream)
{
    CDDT_RANGE("cddt_rm_calc_range_many", stream);
    if (!R || n < 0 || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_rm_calc_range_many");
    if (n == 0) return CDDT_OK;
    cddt::rm_kernel<<<cddt::grid_cap(n, 256, 64), 256, 0, (cudaStream_t)stream>>>(
        R->dist, R->W, R->H, pose_dev, range_dev, steps_dev, n, R->max_range);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

}  // extern "C"
