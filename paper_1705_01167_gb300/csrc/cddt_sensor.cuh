// cddt_sensor.cuh -- device code of the fused sensor model (Section VI):
// per-particle traversal slots, the single-filter kernel and the persistent
// batched kernel.  Included by the sensor and batched translation units,
// which instantiate the kernels, and by cddt_query.cu for the shared types.
#pragma once
#include <cuda_runtime.h>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

enum { MODE_FWD = 0, MODE_BWD = 1, MODE_FWDBWD = 2, MODE_WORK = 3 };

// Work figures of one particle's traversal slot (MODE_WORK).
struct WorkAcc {
    unsigned long long trav = 0, beams = 0, nonempty = 0, probes = 0, paired = 0, sectors = 0;
};

__device__ __forceinline__ int ceil_log2p1(int kb)
{
    // ceil(log2(kb + 1)) for kb >= 0
    return kb <= 0 ? 0 : 32 - __clz((unsigned)kb);
}

// 32-byte sectors a binary search of a sorted CSR bin of kb keys touches
// (kps keys per sector): one for the bin's two offsets, one per probe while
// the remaining range spans more than a sector, one for the last sector.
__device__ __forceinline__ int sorted_sectors(int kb, int kps)
{
    if (kb <= 0) return 1;
    int r = kb, c = 0;
    while (r > kps) {
        r = (r + 1) >> 1;
        ++c;
    }
    return 2 + c;
}

// One particle's beams in traversal slots t = lane, lane + TPP, ... ; smem
// holds one float4 {phi, z, s_lz, c_mr} per beam.  acc sums log2 p.
// m and bc are read where they lie (kernel parameters or shared memory); the
// particle's pose (x, y, th) is held in registers, ranges (forward mode,
// optional) go to `ranges`.
template <typename KT, int MODE, int SEARCH>
__device__ __forceinline__ void particle_slots_at(const MapView &m, const BeamConsts &bc, int B, int D, float x,
                                                  float y, float th, float *ranges, const float *sh, int64_t p,
                                                  bool valid, int lane, int TPP, uint64_t pol, float &acc,
                                                  float &gx, float &gy, WorkAcc &w, bool &ok_out)
{
    const int T = D > 0 ? D : B;
    const bool ok = valid && free_cell(m.grid, m.W, m.H, x, y);
    ok_out = ok;
    const float4 *bt = reinterpret_cast<const float4 *>(sh);
    for (int t = lane; t < T; t += TPP) {
        const int i = t;
        const int j = (D > 0 && t + D < B) ? t + D : -1;
        Cast ci, cj;
        ci.r = cj.r = 0.0f;
        ci.dzx = ci.dzy = cj.dzx = cj.dzy = 0.0f;
        ci.kb = cj.kb = -1;
        bool pairdone = false;
        if (ok) {
            int ki = 0, kj = 0;
            bool vi = query_dir(__fadd_rn(th, sh[4 * i]), m.inv_step, m.N, ki);
            bool vj = j >= 0 && query_dir(__fadd_rn(th, sh[4 * j]), m.inv_step, m.N, kj);
            int kopp = ki + m.S;
            kopp -= (kopp >= m.N) ? m.N : 0;
            if (vj && vi && kj == kopp) {
                Cast f, b;
                bool kf;
                cast_pair<KT, SEARCH>(m, x, y, ki, true, pol, f, b, kf);
                ci = kf ? f : b;
                cj = kf ? b : f;
                pairdone = true;
            } else {
                if (vi) {
                    Cast f, b;
                    bool kf;
                    cast_pair<KT, SEARCH>(m, x, y, ki, false, pol, f, b, kf);
                    ci = kf ? f : b;
                }
                if (vj) {
                    Cast f, b;
                    bool kf;
                    cast_pair<KT, SEARCH>(m, x, y, kj, false, pol, f, b, kf);
                    cj = kf ? f : b;
                }
            }
        }
        if (MODE == MODE_WORK) {
            if (ci.kb >= 0) {
                w.beams++;
                w.trav++;
                w.nonempty += ci.kb > 0;
                w.probes += ceil_log2p1(ci.kb);
                w.sectors += sorted_sectors(ci.kb, 32 / (int)sizeof(KT));
            }
            if (j >= 0 && cj.kb >= 0) {
                w.beams++;
                if (pairdone) w.paired++;
                else {
                    w.trav++;
                    w.nonempty += cj.kb > 0;
                    w.probes += ceil_log2p1(cj.kb);
                    w.sectors += sorted_sectors(cj.kb, 32 / (int)sizeof(KT));
                }
            }
            continue;
        }
        {
            const float4 q = bt[i];
            BeamObs o;
            o.z = q.y;
            o.s_lz = q.z;
            o.c_mr = q.w;
            float dl = 0.f;
            float lp = beam_log2p<MODE != MODE_FWD>(bc, o, ci.r, dl);
            acc += lp;
            if (MODE != MODE_FWD) { gx += dl * ci.dzx; gy += dl * ci.dzy; }
            if (MODE == MODE_FWD && ranges && valid) ranges[p * B + i] = ci.r;
        }
        if (j >= 0) {
            const float4 q = bt[j];
            BeamObs o;
            o.z = q.y;
            o.s_lz = q.z;
            o.c_mr = q.w;
            float dl = 0.f;
            float lp = beam_log2p<MODE != MODE_FWD>(bc, o, cj.r, dl);
            acc += lp;
            if (MODE != MODE_FWD) { gx += dl * cj.dzx; gy += dl * cj.dzy; }
            if (MODE == MODE_FWD && ranges && valid) ranges[p * B + j] = cj.r;
        }
    }
}

// The same with the pose read from part[3 p .. 3 p + 2].
template <typename KT, int MODE, int SEARCH>
__device__ __forceinline__ void particle_slots(const MapView &m, const BeamConsts &bc, int B, int D,
                                               const float *part, float *ranges, const float *sh, int64_t p,
                                               bool valid, int lane, int TPP, uint64_t pol, float &acc, float &gx,
                                               float &gy, WorkAcc &w, bool &ok_out)
{
    float x = 0.f, y = 0.f, th = 0.f;
    if (valid) {
        x = __ldg(part + 3 * p);
        y = __ldg(part + 3 * p + 1);
        th = __ldg(part + 3 * p + 2);
    }
    particle_slots_at<KT, MODE, SEARCH>(m, bc, B, D, x, y, th, ranges, sh, p, valid, lane, TPP, pol, acc, gx, gy,
                                        w, ok_out);
}

__device__ __forceinline__ void stage_beams(const BeamConsts &bc, int B, const float *obs, const float *beam_off,
                                            float *sh)
{
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        BeamObs o = beam_obs(bc, __ldg(obs + i));
        reinterpret_cast<float4 *>(sh)[i] = make_float4(__ldg(beam_off + i), o.z, o.s_lz, o.c_mr);
    }
}

template <int TPP>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void write_particle(const SensorArgs &a, int MODE, int64_t p, float acc, float gx,
                                               float gy)
{
    if (MODE == MODE_FWD || MODE == MODE_FWDBWD) a.logw[p] = acc * kLn2;
    if (MODE == MODE_BWD) {
        float gl = __ldg(a.grad_logw + p);
        a.grad_xy[2 * p] = gl * gx;
        a.grad_xy[2 * p + 1] = gl * gy;
    }
    if (MODE == MODE_FWDBWD) {
        a.grad_xy[2 * p] = gx;
        a.grad_xy[2 * p + 1] = gy;
    }
}

template <typename KT, int MODE, int TPP, int SEARCH>
__global__ void __launch_bounds__(256, 6) sensor_kernel(MapView m, SensorArgs a)
{
    extern __shared__ __align__(16) float sh[];
    stage_beams(a.bc, a.B, a.obs, a.beam_off, sh);
    __syncthreads();
    const uint64_t pol = policy_evict_last();
    const int lane = threadIdx.x % TPP;
    const int group = threadIdx.x / TPP;
    const int ppb = blockDim.x / TPP;
    WorkAcc w;
    unsigned long long passed = 0;
    for (int64_t pb = (int64_t)blockIdx.x * ppb; pb < a.P; pb += (int64_t)gridDim.x * ppb) {
        const int64_t p = pb + group;
        const bool valid = p < a.P;
        float acc = 0.f, gx = 0.f, gy = 0.f;
        bool ok;
        particle_slots<KT, MODE, SEARCH>(m, a.bc, a.B, a.D, a.part, a.ranges, sh, p, valid, lane, TPP, pol, acc,
                                         gx, gy, w, ok);
        if (MODE == MODE_WORK) {
            passed += (ok && lane == 0);
            continue;
        }
        acc = group_sum<TPP>(acc);
        if (MODE != MODE_FWD) {
            gx = group_sum<TPP>(gx);
            gy = group_sum<TPP>(gy);
        }
        if (lane == 0 && valid) write_particle(a, MODE, p, acc, gx, gy);
    }
    if (MODE == MODE_WORK) {
        unsigned long long v[7] = {w.trav, w.beams, w.nonempty, w.probes, w.paired, passed, w.sectors};
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            unsigned long long s = v[q];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) == 0 && s) atomicAdd(a.work + q, s);
        }
    }
}

// ------------------------------------------------------------ batched

struct __align__(16) FilterDev {
    MapView m;
    SensorArgs a;
    int32_t key_u16;
    int32_t pad[3];
};

// What the traversal loop reads of a filter, passed to the batched kernel as
// a __grid_constant__ parameter: reads go through the constant cache (LDC)
// rather than the L1 data path, which the tree searches keep busy.
struct HotFilter {
    MapView m;
    BeamConsts bc;
    int32_t B, D;
};
constexpr int kHotMax = CDDT_CHECKED ? 180 : 220;  // filters per batched launch (parameter space)
struct HotTable {
    HotFilter f[kHotMax];
};
static_assert(sizeof(HotTable) + 512 <= 32764, "kernel parameters are limited to 32764 bytes");

struct WorkItem {
    int32_t filter;  // index into the plan's filters
    int32_t count;
    int64_t first;
    int32_t hot;     // index into the launch's HotTable
    int32_t pad;
};

// Persistent batched sensor model: blocks take (filter, particle range)
// items from an atomic queue until it is empty.  No block waits on another.
// WARPS caps registers so that WARPS warps stay resident per SM (32 leaves
// the compiler its natural 64 registers; 48 trades a few spills for
// occupancy).  One launch serves the filters of one key type (a contiguous
// item range).
template <typename KT, int SEARCH, int TPP, int BLOCK, int WARPS>
__global__ void __launch_bounds__(BLOCK, WARPS * 32 / BLOCK)
    batched_kernel(const __grid_constant__ HotTable tab, const FilterDev *filters, const WorkItem *items,
                   int64_t n_items, unsigned long long *queue, int32_t max_B)
{
    extern __shared__ __align__(16) float sh[];
    __shared__ long long cur;
    // the current item's filter descriptor, read by every thread from shared
    // memory (uniform loads) instead of being held in registers
    __shared__ __align__(16) FilterDev F;
    const uint64_t pol = policy_evict_last();
    const int lane = threadIdx.x % TPP;
    const int group = threadIdx.x / TPP;
    const int ppb = blockDim.x / TPP;
    constexpr int kWords = (int)(sizeof(FilterDev) / sizeof(int4));
    static_assert(sizeof(FilterDev) % sizeof(int4) == 0, "FilterDev must be a multiple of 16 bytes");
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
        WorkAcc w;
        for (int64_t pb = wi.first; pb < wi.first + wi.count; pb += ppb) {
            const int64_t p = pb + group;
            const bool valid = p < wi.first + wi.count;
            float acc = 0.f, gx = 0.f, gy = 0.f;
            bool ok;
            particle_slots<KT, MODE_FWD, SEARCH>(H.m, H.bc, H.B, H.D, F.a.part, nullptr, sh, p, valid, lane, TPP,
                                                 pol, acc, gx, gy, w, ok);
            acc = group_sum<TPP>(acc);
            if (lane == 0 && valid) F.a.logw[p] = acc * kLn2;
        }
        __syncthreads();
    }
    (void)max_B;
}

inline size_t beam_smem(int B) { return sizeof(float) * 4 * (size_t)B; }

// One step of gradient pose refinement: (x, y) += eta g / max(|g|, 1e-12),
// every operation correctly rounded in this order (no contraction).
__device__ __forceinline__ void refine_move(float &x, float &y, float gx, float gy, float eta)
{
    const float n = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
    const float s = __fdiv_rn(eta, fmaxf(n, 1e-12f));
    x = __fadd_rn(x, __fmul_rn(gx, s));
    y = __fadd_rn(y, __fmul_rn(gy, s));
}

// Gradient pose refinement of a plan's filters in one persistent launch (the
// differentiation extension): every particle keeps its pose in registers
// and, `steps` times, evaluates log w and g = d log w / d(x, y) at the pose
// (the forward and adjoint traversal of the sensor model, one pass) and
// moves by refine_move; then it evaluates once more.  Written per particle:
// the final log w, the final g and the refined pose (theta unchanged).  TPP
// lanes share a particle's traversal slots and their sums (butterfly
// shuffles, so every lane holds the same g and takes the same step).  Items
// (filter, particle range of blockDim.x / TPP) come from an atomic queue;
// no block waits on another.
template <typename KT, int TPP>
__global__ void __launch_bounds__(256, 4)
    refine_kernel(const __grid_constant__ HotTable tab, const FilterDev *filters, const WorkItem *items,
                  int64_t n_items, unsigned long long *queue, int32_t steps, float eta)
{
    extern __shared__ __align__(16) float sh[];
    __shared__ long long cur;
    __shared__ __align__(16) FilterDev F;
    const uint64_t pol = policy_evict_last();
    const int lane = threadIdx.x % TPP;
    const int group = threadIdx.x / TPP;
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
            acc = group_sum<TPP>(acc);
            gx = group_sum<TPP>(gx);
            gy = group_sum<TPP>(gy);
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

typedef void (*RefineFn)(const HotTable, const FilterDev *, const WorkItem *, int64_t, unsigned long long *,
                         int32_t, float);

template <typename KT>
inline RefineFn refine_fn_kt(int tpp)
{
    switch (tpp) {
    case 1: return refine_kernel<KT, 1>;
    case 2: return refine_kernel<KT, 2>;
    case 4: return refine_kernel<KT, 4>;
    case 8: return refine_kernel<KT, 8>;
    case 16: return refine_kernel<KT, 16>;
    case 32: return refine_kernel<KT, 32>;
    default: return nullptr;
    }
}

// Kernel pointer of the refinement kernel for a key type and lanes per
// particle (cddt_refine.cu); nullptr for an unknown tpp.
RefineFn refine_fn(bool u16, int tpp);

typedef void (*BatchedFn)(const HotTable, const FilterDev *, const WorkItem *, int64_t, unsigned long long *,
                          int32_t);

// Kernel pointer of the batched kernel for a key type and launch shape
// (cddt_batched_f32.cu, cddt_batched_u16.cu); nullptr for an unknown shape.
BatchedFn batched_fn_f32(int search, int tpp, int block, int regcap);
BatchedFn batched_fn_u16(int search, int tpp, int block, int regcap);

// Single-filter sensor launches (cddt_sensor_f32.cu, cddt_sensor_u16.cu).
// Tree layout, every mode; the binary-search layout for the forward mode only
// (it gives the same answers, so the other modes always use the tree).
cddt_status launch_sensor_f32(const cddt_s *h, const SensorArgs &a, int mode, int tpp, int threads, cudaStream_t st);
cddt_status launch_sensor_u16(const cddt_s *h, const SensorArgs &a, int mode, int tpp, int threads, cudaStream_t st);
cddt_status launch_sensor_binary(const cddt_s *h, const SensorArgs &a, int tpp, int threads, cudaStream_t st);

template <typename KT, int MODE, int SEARCH>
inline cddt_status launch_sensor_tpp(const cddt_s *h, const SensorArgs &a, int tpp, int threads, cudaStream_t st)
{
    MapView m = h->view();
    int ppb = threads / tpp;
    int64_t blocks = (a.P + ppb - 1) / ppb;
    if (blocks > (int64_t)sm_count() * 32) blocks = (int64_t)sm_count() * 32;
    if (blocks < 1) blocks = 1;
    size_t sm = beam_smem(a.B);
    void (*fn)(MapView, SensorArgs) = nullptr;
    switch (tpp) {
    case 1: fn = sensor_kernel<KT, MODE, 1, SEARCH>; break;
    case 2: fn = sensor_kernel<KT, MODE, 2, SEARCH>; break;
    case 4: fn = sensor_kernel<KT, MODE, 4, SEARCH>; break;
    case 8: fn = sensor_kernel<KT, MODE, 8, SEARCH>; break;
    case 16: fn = sensor_kernel<KT, MODE, 16, SEARCH>; break;
    default: fn = sensor_kernel<KT, MODE, 32, SEARCH>; break;
    }
    if (sm > 48 * 1024) CDDT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    fn<<<(unsigned)blocks, threads, sm, st>>>(m, a);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

template <typename KT>
inline cddt_status launch_sensor_mode(const cddt_s *h, const SensorArgs &a, int mode, int tpp, int threads,
                                      cudaStream_t st)
{
    switch (mode) {
    case MODE_FWD: return launch_sensor_tpp<KT, MODE_FWD, CDDT_SEARCH_TREE>(h, a, tpp, threads, st);
    case MODE_BWD: return launch_sensor_tpp<KT, MODE_BWD, CDDT_SEARCH_TREE>(h, a, tpp, threads, st);
    case MODE_FWDBWD: return launch_sensor_tpp<KT, MODE_FWDBWD, CDDT_SEARCH_TREE>(h, a, tpp, threads, st);
    default: return launch_sensor_tpp<KT, MODE_WORK, CDDT_SEARCH_TREE>(h, a, tpp, threads, st);
    }
}

template <typename KT, int SEARCH, int WARPS>
inline BatchedFn batched_fn_kt(int tpp, int block)
{
#define CDDT_BF(T, B) if (tpp == T && block == B) return batched_kernel<KT, SEARCH, T, B, WARPS>;
    CDDT_BF(1, 256) CDDT_BF(1, 512)
    CDDT_BF(2, 256) CDDT_BF(2, 512)
    CDDT_BF(4, 256) CDDT_BF(4, 512)
    CDDT_BF(8, 256) CDDT_BF(8, 512)
#undef CDDT_BF
    return nullptr;
}

// 16 and 32 lanes per particle, for plans with few particles (their own
// translation units, cddt_batched_wide_*.cu, to keep compile times short).
template <typename KT, int SEARCH, int WARPS>
inline BatchedFn batched_fn_kt_wide(int tpp, int block)
{
#define CDDT_BF(T, B) if (tpp == T && block == B) return batched_kernel<KT, SEARCH, T, B, WARPS>;
    CDDT_BF(16, 256) CDDT_BF(16, 512)
    CDDT_BF(32, 256) CDDT_BF(32, 512)
#undef CDDT_BF
    return nullptr;
}
BatchedFn batched_fn_wide_f32(int search, int tpp, int block, int regcap);
BatchedFn batched_fn_wide_u16(int search, int tpp, int block, int regcap);

}  // namespace cddt
