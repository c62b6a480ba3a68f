// cddt_refine.cu -- the plan's gradient pose refinement kernels (both key
// types, every lanes-per-particle count).  Up to one warp per particle the
// kernel is refine_kernel (cddt_sensor.cuh); wider particles are below.
#include "cddt_sensor.cuh"

namespace cddt {

// refine_kernel for TPP = 64, 128 or 256 lanes per particle (TPP / 32 warps
// of the block): plans with few particles, whose particles then have more
// lanes to split their traversal slots over.  Each evaluation's sums are
// taken warp by warp (butterfly shuffles), then across the particle's warps
// through shared memory in warp order, so every lane of the particle holds
// the same sums and takes the same step; the two halves of `red` alternate
// between evaluations, so one barrier per evaluation suffices.
template <typename KT, int TPP>
__global__ void __launch_bounds__(kRefineBlock, 4)
    refine_kernel_wide(const __grid_constant__ HotTable tab, const FilterDev *filters, const WorkItem *items,
                       int64_t n_items, unsigned long long *queue, int32_t steps, float eta)
{
    static_assert(TPP % 32 == 0 && TPP <= kRefineBlock, "whole warps of one block per particle");
    constexpr int WPP = TPP / 32;
    extern __shared__ __align__(16) float sh[];
    __shared__ long long cur;
    __shared__ __align__(16) FilterDev F;
    __shared__ float red[2][kRefineBlock / 32][3];
    const uint64_t pol = policy_evict_last();
    const int lane = threadIdx.x % TPP;
    const int group = threadIdx.x / TPP;
    const int warp = threadIdx.x >> 5;
    constexpr int kWords = (int)(sizeof(FilterDev) / sizeof(int4));
    for (;;) {
        if (threadIdx.x == 0) cur = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long it = cur;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        for (int q = threadIdx.x; q < kWords; q += blockDim.x)
            reinterpret_cast<int4 *>(&F)[q] = reinterpret_cast<const int4 *>(filters + wi.filter)[q];
        __syncthreads();
        const HotFilter &H = tab.f[wi.hot];
        stage_beams(H.bc, H.B, F.a.obs, F.a.beam_off, sh);
        __syncthreads();
        const int64_t p = wi.first + group;
        const bool valid = group < wi.count;
        float x = 0.f, y = 0.f, th = 0.f;
        if (valid) {
            x = __ldg(F.a.part + 3 * p);
            y = __ldg(F.a.part + 3 * p + 1);
            th = __ldg(F.a.part + 3 * p + 2);
        }
        WorkAcc w;
        float acc = 0.f, gx = 0.f, gy = 0.f;
        for (int s = 0; s <= steps; ++s) {
            acc = gx = gy = 0.f;
            bool ok;
            particle_slots_at<KT, MODE_FWDBWD, CDDT_SEARCH_TREE>(H.m, H.bc, H.B, H.D, x, y, th, nullptr, sh, p,
                                                                 valid, lane, TPP, pol, acc, gx, gy, w, ok);
            acc = group_sum<32>(acc);
            gx = group_sum<32>(gx);
            gy = group_sum<32>(gy);
            float(*r)[3] = red[s & 1];
            if ((threadIdx.x & 31) == 0) {
                r[warp][0] = acc;
                r[warp][1] = gx;
                r[warp][2] = gy;
            }
            __syncthreads();
            acc = gx = gy = 0.f;
#pragma unroll
            for (int k = 0; k < WPP; ++k) {
                acc += r[group * WPP + k][0];
                gx += r[group * WPP + k][1];
                gy += r[group * WPP + k][2];
            }
            if (s < steps) refine_move(x, y, gx, gy, eta);
        }
        if (lane == 0 && valid) {
            F.a.logw[p] = acc * kLn2;
            F.a.grad_xy[2 * p] = gx;
            F.a.grad_xy[2 * p + 1] = gy;
            F.a.part_out[3 * p] = x;
            F.a.part_out[3 * p + 1] = y;
            F.a.part_out[3 * p + 2] = th;
        }
        __syncthreads();
    }
}

template <typename KT>
static RefineFn refine_fn_any(int tpp)
{
    switch (tpp) {
    case 64: return refine_kernel_wide<KT, 64>;
    case 128: return refine_kernel_wide<KT, 128>;
    case 256: return refine_kernel_wide<KT, 256>;
    default: return refine_fn_kt<KT>(tpp);
    }
}

RefineFn refine_fn(bool u16, int tpp) { return u16 ? refine_fn_any<uint16_t>(tpp) : refine_fn_any<float>(tpp); }

}  // namespace cddt
