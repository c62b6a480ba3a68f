// cddt_mcl.cu -- the particle filter steps around the sensor model
// (Section I): the odometry motion model before it and low-variance
// resampling after it, for many filters (segments of one particle array) in
// one launch each.
#include <cuda_runtime.h>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

namespace cddt {

// Segment (filter) of particle p: the last f with seg[f] <= p.
__device__ __forceinline__ int segment_of(const int64_t *seg, int F, int64_t p)
{
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seg + mid) <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr float kTwoPi = 6.28318530717958647692f;

// Odometry motion model: the robot moved (dx, dy) in its own frame and
// turned by dth; particle p applies that increment plus its noise sample
// (nx, ny, nth): x += a cos(th) - b sin(th), y += a sin(th) + b cos(th) with
// a = dx + nx, b = dy + ny, then th += dth + nth wrapped into [0, 2 pi) by
// one add or subtract of 2 pi.
__global__ void motion_kernel(float *part, int64_t P, const int64_t *seg, int F, const float *odom,
                              const float *noise)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int f = segment_of(seg, F, p);
        const float x = part[3 * p], y = part[3 * p + 1], th = part[3 * p + 2];
        const float a = __fadd_rn(__ldg(odom + 3 * f), __ldg(noise + 3 * p));
        const float b = __fadd_rn(__ldg(odom + 3 * f + 1), __ldg(noise + 3 * p + 1));
        float s, c;
        sincosf(th, &s, &c);
        const float nx = __fadd_rn(x, __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, s)));
        const float ny = __fadd_rn(y, __fadd_rn(__fmul_rn(a, s), __fmul_rn(b, c)));
        float nt = __fadd_rn(th, __fadd_rn(__ldg(odom + 3 * f + 2), __ldg(noise + 3 * p + 2)));
        if (nt >= kTwoPi) nt = __fsub_rn(nt, kTwoPi);
        else if (nt < 0.0f) nt = __fadd_rn(nt, kTwoPi);
        part[3 * p] = nx;
        part[3 * p + 1] = ny;
        part[3 * p + 2] = nt;
    }
}

// Low-variance (systematic) resampling of one filter per block: weights
// w_i = exp(logw_i - max logw) and their running sums C_i in double, then
// output m takes the first input i with C_i > (u0 + m) / P * C_{P-1}.  The
// sums are taken per thread over a contiguous chunk and offset by a scan of
// the chunk totals (a fixed order: the same bits on every run).  Weights
// that exp(logw - max) leaves undefined: when no log-weight is above -inf
// (all -inf or NaN: no particle has weight) every particle weighs 1;
// otherwise a NaN log-weight weighs 0, and when the largest is +inf exactly
// the +inf particles weigh 1.
constexpr int kResampleThreads = 512;

__device__ __forceinline__ double resample_weight(float lw, double m0)
{
    if (m0 == -__builtin_huge_val()) return 1.0;
    if (isnan(lw)) return 0.0;
    if (m0 == __builtin_huge_val()) return lw == __builtin_huge_valf() ? 1.0 : 0.0;
    return exp((double)lw - m0);
}

__global__ void __launch_bounds__(kResampleThreads) resample_kernel(const float *part, const float *logw,
                                                                    const int64_t *seg, const float *u0,
                                                                    float *out, int32_t *index, double *csum)
{
    __shared__ double red[kResampleThreads];
    __shared__ float mx_s;
    const int f = blockIdx.x;
    const int64_t a = seg[f], n = seg[f + 1] - seg[f];
    if (n <= 0) return;
    const float *lw = logw + a;
    double *C = csum + a;
    // max log-weight
    float mx = -__builtin_huge_valf();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, lw[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = -__builtin_huge_valf();
        for (int w = 0; w < kResampleThreads / 32; ++w) m = fmaxf(m, (float)red[w]);
        mx_s = m;
    }
    __syncthreads();
    const double m0 = (double)mx_s;
    // chunk sums, a scan of them, then the running sums
    const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = threadIdx.x * chunk, i1 = min(n, i0 + chunk);
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) {  // the weights wait in C for the running sums
        const double w = resample_weight(lw[i], m0);
        C[i] = w;
        s += w;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const double v = red[t];
            red[t] = acc;
            acc += v;
        }
    }
    __syncthreads();
    double run = red[threadIdx.x];
    for (int64_t i = i0; i < i1; ++i) {
        run += C[i];
        C[i] = run;
    }
    __syncthreads();
    const double total = C[n - 1];
    const double uf = (double)u0[f];
    for (int64_t m = threadIdx.x; m < n; m += blockDim.x) {
        const double target = (uf + (double)m) / (double)n * total;
        int64_t lo = 0, hi = n - 1;  // first i with C_i > target (the last one when none is)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (C[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const float *src = part + 3 * (a + lo);
        out[3 * (a + m)] = src[0];
        out[3 * (a + m) + 1] = src[1];
        out[3 * (a + m) + 2] = src[2];
        if (index) index[a + m] = (int32_t)lo;
    }
}

}  // namespace cddt

extern "C" {

cddt_status cddt_motion(float *particles_dev, int64_t P, const int64_t *seg_start_dev, int32_t F,
                        const float *odom_dev, const float *noise_dev, void *stream)
{
    CDDT_RANGE("cddt_motion", stream);
    if (P < 0 || F < 1 || (P > 0 && (!particles_dev || !seg_start_dev || !odom_dev || !noise_dev)))
        return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_motion");
    if (P == 0) return CDDT_OK;
    cddt::motion_kernel<<<cddt::grid_cap(P, 256, 16), 256, 0, (cudaStream_t)stream>>>(
        particles_dev, P, seg_start_dev, F, odom_dev, noise_dev);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

cddt_status cddt_resample(const float *particles_dev, const float *logw_dev, const int64_t *seg_start_dev,
                          int32_t F, const float *u0_dev, float *out_dev, int32_t *index_dev, double *scratch_dev,
                          void *stream)
{
    CDDT_RANGE("cddt_resample", stream);
    if (F < 1 || !particles_dev || !logw_dev || !seg_start_dev || !u0_dev || !out_dev || !scratch_dev)
        return CDDT_ERR_ARG;
    if (particles_dev == out_dev) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_resample");
    cddt::resample_kernel<<<(unsigned)F, cddt::kResampleThreads, 0, (cudaStream_t)stream>>>(
        particles_dev, logw_dev, seg_start_dev, u0_dev, out_dev, index_dev, scratch_dev);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

}  // extern "C"
