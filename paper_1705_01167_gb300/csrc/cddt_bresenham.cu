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

// Start cell floor(p + 1/2), end cell floor(p + max_range (cos, sin) + 1/2)
// (in double), integer error stepping; the distance from the query point to
// the first occupied cell's centre (double, clamped to max_range); 0 from an
// occupied or off-map cell or for a non-finite heading (as a CDDT query); max_range when the walk leaves the map or ends.
__global__ void bresenham_kernel(const uint8_t *grid, int W, int H, const float *pose, float *out, int64_t n,
                                 double max_range)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        const double fx0 = floor(x + 0.5), fy0 = floor(y + 0.5);
        if (!(fx0 >= 0.0 && fx0 < (double)W && fy0 >= 0.0 && fy0 < (double)H) || !isfinite(th) ||
            __ldg(grid + (int64_t)fy0 * W + (int64_t)fx0)) {
            out[q] = 0.0f;
            continue;
        }
        double s, c;
        sincos(th, &s, &c);
        const long long x0 = (long long)fx0, y0 = (long long)fy0;
        const long long x1 = (long long)floor(x + max_range * c + 0.5);
        const long long y1 = (long long)floor(y + max_range * s + 0.5);
        const long long ddx = llabs(x1 - x0), ddy = -llabs(y1 - y0);
        const int sx = x0 < x1 ? 1 : -1, sy = y0 < y1 ? 1 : -1;
        long long err = ddx + ddy, cx = x0, cy = y0;
        double res = max_range;
        while (!(cx == x1 && cy == y1)) {
            const long long e2 = 2 * err;
            if (e2 >= ddy) { err += ddy; cx += sx; }
            if (e2 <= ddx) { err += ddx; cy += sy; }
            if (cx < 0 || cx >= W || cy < 0 || cy >= H) break;
            if (__ldg(grid + cy * W + cx)) {
                const double dx = (double)cx - x, dy = (double)cy - y;
                res = fmin(sqrt(dx * dx + dy * dy), max_range);
                break;
            }
        }
        out[q] = (float)res;
    }
}

}  // namespace cddt

extern "C" cddt_status cddt_cast_bresenham(cddt_t h, const float *pose_dev, float *range_dev, int64_t n, void *stream)
{
    CDDT_RANGE("cddt_cast_bresenham");
    if (!h || n < 0 || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_cast_bresenham");
    if (n == 0) return CDDT_OK;
    cddt::bresenham_kernel<<<cddt::grid_cap(n, 256, 152 * 64), 256, 0, (cudaStream_t)stream>>>(
        h->grid, h->W, h->H, pose_dev, range_dev, n, (double)h->max_range);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}
