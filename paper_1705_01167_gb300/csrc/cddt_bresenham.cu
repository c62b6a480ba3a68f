// cddt_bresenham.cu -- the Bresenham line caster (Section II, the paper's
// "BL" baseline): walk the grid cells on the digital line from the query's
// cell towards its max-range end point and stop at the first occupied one.
// A second baseline family beside the CDDT, one thread per ray.
#include <cuda_runtime.h>

#include <cmath>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

namespace cddt {

// Integer error stepping from (x0, y0) to (x1, y1) (the textbook all-octant
// form); returns the first occupied cell met in (hx, hy), false when the
// walk leaves the map or reaches its end.  I is int when every error term
// fits in 32 bits, else long long: the cells visited are the same.
template <typename I>
__device__ __forceinline__ bool bresenham_walk(const uint8_t *grid, int W, int H, I x0, I y0, I x1, I y1, int &hx,
                                               int &hy)
{
    const I ddx = x1 > x0 ? x1 - x0 : x0 - x1, ddy = -(y1 > y0 ? y1 - y0 : y0 - y1);
    const I sx = x0 < x1 ? 1 : -1, sy = y0 < y1 ? 1 : -1;
    I err = ddx + ddy, cx = x0, cy = y0;
    while (!(cx == x1 && cy == y1)) {
        const I e2 = 2 * err;
        if (e2 >= ddy) { err += ddy; cx += sx; }
        if (e2 <= ddx) { err += ddx; cy += sy; }
        if (cx < 0 || cx >= W || cy < 0 || cy >= H) return false;
        if (__ldg(grid + (int64_t)cy * W + cx)) {
            hx = (int)cx;
            hy = (int)cy;
            return true;
        }
    }
    return false;
}

// Start cell floor(p + 1/2), end cell floor(fma(max_range, (c, s), p) + 1/2)
// with c, s = dir_sincos(theta) (reading D1), all float32; the distance from
// the query point to the first occupied cell's centre (float32, clamped to
// max_range); 0 from an occupied or off-map cell or for a non-finite
// coordinate (as a CDDT query); max_range when the walk leaves the map or
// ends.
__global__ void bresenham_kernel(const uint8_t *grid, int W, int H, const float *pose, float *out, int64_t n,
                                 float max_range)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        const float fx0 = floorf(__fadd_rn(x, 0.5f)), fy0 = floorf(__fadd_rn(y, 0.5f));
        if (!(isfinite(x) && isfinite(y) && isfinite(th)) ||
            !(fx0 >= 0.0f && fx0 < (float)W && fy0 >= 0.0f && fy0 < (float)H) ||
            __ldg(grid + (int64_t)fy0 * W + (int64_t)fx0)) {
            out[q] = 0.0f;
            continue;
        }
        float s, c;
        dir_sincos(th, s, c);
        const float fx1 = floorf(__fadd_rn(__fmaf_rn(max_range, c, x), 0.5f));
        const float fy1 = floorf(__fadd_rn(__fmaf_rn(max_range, s, y), 0.5f));
        int hx = 0, hy = 0;
        bool hit;
        if (fabsf(fx1) < 1e9f && fabsf(fy1) < 1e9f)  // |error terms| < 2^31
            hit = bresenham_walk<int>(grid, W, H, (int)fx0, (int)fy0, (int)fx1, (int)fy1, hx, hy);
        else
            hit = bresenham_walk<long long>(grid, W, H, (long long)fx0, (long long)fy0, (long long)fx1,
                                            (long long)fy1, hx, hy);
        float res = max_range;
        if (hit) {
            const float dx = __fsub_rn((float)hx, x), dy = __fsub_rn((float)hy, y);
            res = fminf(__fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))), max_range);
        }
        out[q] = res;
    }
}

}  // namespace cddt

extern "C" cddt_status cddt_cast_bresenham(cddt_t h, const float *pose_dev, float *range_dev, int64_t n, void *stream)
{
    CDDT_RANGE("cddt_cast_bresenham", stream);
    if (!h || n < 0 || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_cast_bresenham");
    if (n == 0) return CDDT_OK;
    cddt::bresenham_kernel<<<cddt::grid_cap(n, 256, 64), 256, 0, (cudaStream_t)stream>>>(
        h->grid, h->W, h->H, pose_dev, range_dev, n, h->max_range);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}
