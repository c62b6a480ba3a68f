// cddt_query.cu -- ray casting and the fused beam sensor model on the GPU.
//
// Ray cast (Section IV-B): project the query into its slice, pick the bin,
// find the nearest zero point beyond x' (successor; predecessor for the
// theta + pi half of the circle, Section IV-C), return the distance.  The
// sensor model (Section VI) casts every beam of a particle, evaluates the
// beam-model mixture and sums log p over the beams.  Beams i and i + D that
// point opposite ways and fall on the same stored slice share one search
// (Section IV-C, "index i - 1").
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

// ------------------------------------------------------------ single ray

template <typename KT>
__device__ __forceinline__ Cast cast_one(const MapView &m, float x, float y, float th)
{
    Cast r;
    r.r = 0.0f;
    r.dzx = r.dzy = 0.0f;
    r.kb = -1;
    if (!free_cell(m.grid, m.W, m.H, x, y)) return r;
    int k;
    if (!query_dir(th, m.inv_step, m.N, k)) return r;
    Cast f, b;
    bool kf;
    cast_pair<KT>(m, x, y, k, false, f, b, kf);
    return kf ? f : b;
}

template <typename KT>
__global__ void calc_range_kernel(MapView m, const float *pose, float *out, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        float x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        out[q] = cast_one<KT>(m, x, y, th).r;
    }
}

// Slice bucket of a query: its stored slice, or S when no search is needed.
__device__ __forceinline__ int slice_bucket(const MapView &m, float x, float y, float th)
{
    if (!free_cell(m.grid, m.W, m.H, x, y)) return m.S;
    int k;
    if (!query_dir(th, m.inv_step, m.N, k)) return m.S;
    return k >= m.S ? k - m.S : k;
}

__global__ void bucket_kernel(MapView m, const float *pose, int64_t n, uint32_t *bucket, uint32_t *hist)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int b = slice_bucket(m, __ldg(pose + 3 * q), __ldg(pose + 3 * q + 1), __ldg(pose + 3 * q + 2));
        bucket[q] = (uint32_t)b;
        unsigned peers = __match_any_sync(__activemask(), b);
        int leader = __ffs(peers) - 1;
        if ((threadIdx.x & 31) == leader) atomicAdd(hist + b, (uint32_t)__popc(peers));
    }
}

__global__ void place_kernel(const uint32_t *bucket, int64_t n, uint32_t *cursor, uint32_t *perm)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = bucket[q];
        unsigned peers = __match_any_sync(__activemask(), b);
        int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(cursor + b, (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        perm[base + __popc(peers & ((1u << lane) - 1))] = (uint32_t)q;
    }
}

template <typename KT>
__global__ void calc_range_sorted_kernel(MapView m, const float *pose, const uint32_t *perm, float *out,
                                         int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q = perm[i];
        float x = __ldg(pose + 3 * (int64_t)q), y = __ldg(pose + 3 * (int64_t)q + 1),
              th = __ldg(pose + 3 * (int64_t)q + 2);
        out[q] = cast_one<KT>(m, x, y, th).r;
    }
}

// ------------------------------------------------------------ sensor model

enum { MODE_FWD = 0, MODE_BWD = 1, MODE_FWDBWD = 2, MODE_WORK = 3 };

// Work figures of one particle's traversal slot (MODE_WORK).
struct WorkAcc {
    unsigned long long trav = 0, beams = 0, nonempty = 0, probes = 0, paired = 0;
};

__device__ __forceinline__ int ceil_log2p1(int kb)
{
    // ceil(log2(kb + 1)) for kb >= 0
    return kb <= 0 ? 0 : 32 - __clz((unsigned)kb);
}

// One particle's beams in traversal slots t = lane, lane + TPP, ... ; smem
// holds phi[B], z[B], e_lz[B], c_mr[B].
template <typename KT, int MODE>
__device__ __forceinline__ void particle_slots(const MapView &m, const SensorArgs &a, const float *sh,
                                               int64_t p, bool valid, int lane, int TPP, float &acc,
                                               float &gx, float &gy, WorkAcc &w, bool &ok_out)
{
    const int B = a.B, D = a.D;
    const int T = D > 0 ? D : B;
    float x = 0.f, y = 0.f, th = 0.f;
    if (valid) {
        x = __ldg(a.part + 3 * p);
        y = __ldg(a.part + 3 * p + 1);
        th = __ldg(a.part + 3 * p + 2);
    }
    const bool ok = valid && free_cell(m.grid, m.W, m.H, x, y);
    ok_out = ok;
    const float *phi = sh, *zz = sh + B, *elz = sh + 2 * B, *cmr = sh + 3 * B;
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
            bool vi = query_dir(__fadd_rn(th, phi[i]), m.inv_step, m.N, ki);
            bool vj = j >= 0 && query_dir(__fadd_rn(th, phi[j]), m.inv_step, m.N, kj);
            if (vj && vi && kj == (ki + m.S) % m.N) {
                Cast f, b;
                bool kf;
                cast_pair<KT>(m, x, y, ki, true, f, b, kf);
                ci = kf ? f : b;
                cj = kf ? b : f;
                pairdone = true;
            } else {
                if (vi) {
                    Cast f, b;
                    bool kf;
                    cast_pair<KT>(m, x, y, ki, false, f, b, kf);
                    ci = kf ? f : b;
                }
                if (vj) {
                    Cast f, b;
                    bool kf;
                    cast_pair<KT>(m, x, y, kj, false, f, b, kf);
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
            }
            if (j >= 0 && cj.kb >= 0) {
                w.beams++;
                if (pairdone) w.paired++;
                else {
                    w.trav++;
                    w.nonempty += cj.kb > 0;
                    w.probes += ceil_log2p1(cj.kb);
                }
            }
            continue;
        }
        {
            BeamObs o;
            o.z = zz[i];
            o.e_lz = elz[i];
            o.c_mr = cmr[i];
            float dl = 0.f;
            float lp = beam_logp<MODE != MODE_FWD>(a.bc, o, ci.r, dl);
            acc += lp;
            if (MODE != MODE_FWD) { gx += dl * ci.dzx; gy += dl * ci.dzy; }
            if (MODE == MODE_FWD && a.ranges && valid) a.ranges[p * B + i] = ci.r;
        }
        if (j >= 0) {
            BeamObs o;
            o.z = zz[j];
            o.e_lz = elz[j];
            o.c_mr = cmr[j];
            float dl = 0.f;
            float lp = beam_logp<MODE != MODE_FWD>(a.bc, o, cj.r, dl);
            acc += lp;
            if (MODE != MODE_FWD) { gx += dl * cj.dzx; gy += dl * cj.dzy; }
            if (MODE == MODE_FWD && a.ranges && valid) a.ranges[p * B + j] = cj.r;
        }
    }
}

__device__ __forceinline__ void stage_beams(const SensorArgs &a, float *sh)
{
    for (int i = threadIdx.x; i < a.B; i += blockDim.x) {
        BeamObs o = beam_obs(a.bc, __ldg(a.obs + i));
        sh[i] = __ldg(a.beam_off + i);
        sh[a.B + i] = o.z;
        sh[2 * a.B + i] = o.e_lz;
        sh[3 * a.B + i] = o.c_mr;
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
    if (MODE == MODE_FWD || MODE == MODE_FWDBWD) a.logw[p] = acc;
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

template <typename KT, int MODE, int TPP>
__global__ void sensor_kernel(MapView m, SensorArgs a)
{
    extern __shared__ float sh[];
    stage_beams(a, sh);
    __syncthreads();
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
        particle_slots<KT, MODE>(m, a, sh, p, valid, lane, TPP, acc, gx, gy, w, ok);
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
        unsigned long long v[6] = {w.trav, w.beams, w.nonempty, w.probes, w.paired, passed};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            unsigned long long s = v[q];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) == 0 && s) atomicAdd(a.work + q, s);
        }
    }
}

// ------------------------------------------------------------ batched

struct FilterDev {
    MapView m;
    SensorArgs a;
    int32_t key_u16;
};

struct WorkItem {
    int32_t filter;
    int32_t count;
    int64_t first;
};

// Persistent batched sensor model: blocks take (filter, particle range)
// items from an atomic queue until it is empty.  No block waits on another.
template <int TPP>
__global__ void batched_kernel(const FilterDev *filters, const WorkItem *items, int64_t n_items,
                               unsigned long long *queue, int32_t max_B)
{
    extern __shared__ float sh[];
    __shared__ long long cur;
    const int lane = threadIdx.x % TPP;
    const int group = threadIdx.x / TPP;
    const int ppb = blockDim.x / TPP;
    for (;;) {
        if (threadIdx.x == 0) cur = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long it = cur;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        const FilterDev &F = filters[wi.filter];
        const MapView m = F.m;
        const SensorArgs a = F.a;
        stage_beams(a, sh);
        __syncthreads();
        WorkAcc w;
        for (int64_t pb = wi.first; pb < wi.first + wi.count; pb += ppb) {
            const int64_t p = pb + group;
            const bool valid = p < wi.first + wi.count;
            float acc = 0.f, gx = 0.f, gy = 0.f;
            bool ok;
            if (F.key_u16)
                particle_slots<uint16_t, MODE_FWD>(m, a, sh, p, valid, lane, TPP, acc, gx, gy, w, ok);
            else
                particle_slots<float, MODE_FWD>(m, a, sh, p, valid, lane, TPP, acc, gx, gy, w, ok);
            acc = group_sum<TPP>(acc);
            if (lane == 0 && valid) a.logw[p] = acc;
        }
        __syncthreads();
    }
    (void)max_B;
}

// ------------------------------------------------------------ host

static size_t beam_smem(int B) { return sizeof(float) * 4 * (size_t)B; }

template <typename KT, int MODE>
static cddt_status launch_sensor_tpp(const cddt_s *h, const SensorArgs &a, int tpp, int threads, cudaStream_t st)
{
    MapView m = h->view();
    int ppb = threads / tpp;
    int64_t blocks = (a.P + ppb - 1) / ppb;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    size_t sm = beam_smem(a.B);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaSuccess;
        switch (tpp) {
        case 4: e = cudaFuncSetAttribute(sensor_kernel<KT, MODE, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
        case 8: e = cudaFuncSetAttribute(sensor_kernel<KT, MODE, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
        case 16: e = cudaFuncSetAttribute(sensor_kernel<KT, MODE, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
        default: e = cudaFuncSetAttribute(sensor_kernel<KT, MODE, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
        }
        CDDT_CUDA(e);
    }
    switch (tpp) {
    case 4: sensor_kernel<KT, MODE, 4><<<(unsigned)blocks, threads, sm, st>>>(m, a); break;
    case 8: sensor_kernel<KT, MODE, 8><<<(unsigned)blocks, threads, sm, st>>>(m, a); break;
    case 16: sensor_kernel<KT, MODE, 16><<<(unsigned)blocks, threads, sm, st>>>(m, a); break;
    default: sensor_kernel<KT, MODE, 32><<<(unsigned)blocks, threads, sm, st>>>(m, a); break;
    }
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// Threads per particle: enough lanes that each has a few traversal slots.
static int pick_tpp(int B, int D)
{
    int T = D > 0 ? D : B;
    if (T <= 24) return 4;
    if (T <= 96) return 8;
    if (T <= 256) return 16;
    return 32;
}

cddt_status launch_sensor(const cddt_s *h, const SensorArgs &a, int mode, cudaStream_t st)
{
    int tpp = pick_tpp(a.B, a.D);
    int threads = 256;
    if (h->u16) {
        switch (mode) {
        case MODE_FWD: return launch_sensor_tpp<uint16_t, MODE_FWD>(h, a, tpp, threads, st);
        case MODE_BWD: return launch_sensor_tpp<uint16_t, MODE_BWD>(h, a, tpp, threads, st);
        case MODE_FWDBWD: return launch_sensor_tpp<uint16_t, MODE_FWDBWD>(h, a, tpp, threads, st);
        default: return launch_sensor_tpp<uint16_t, MODE_WORK>(h, a, tpp, threads, st);
        }
    }
    switch (mode) {
    case MODE_FWD: return launch_sensor_tpp<float, MODE_FWD>(h, a, tpp, threads, st);
    case MODE_BWD: return launch_sensor_tpp<float, MODE_BWD>(h, a, tpp, threads, st);
    case MODE_FWDBWD: return launch_sensor_tpp<float, MODE_FWDBWD>(h, a, tpp, threads, st);
    default: return launch_sensor_tpp<float, MODE_WORK>(h, a, tpp, threads, st);
    }
}

cddt_status calc_range(cddt_s *h, const float *pose, float *out, int64_t n, int sorted, cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    MapView m = h->view();
    const int threads = 256;
    if (!sorted) {
        unsigned blocks = grid_cap(n, threads, 152 * 64);
        if (h->u16) calc_range_kernel<uint16_t><<<blocks, threads, 0, st>>>(m, pose, out, n);
        else calc_range_kernel<float><<<blocks, threads, 0, st>>>(m, pose, out, n);
        CDDT_CUDA(cudaGetLastError());
        return CDDT_OK;
    }
    if (n > 0xffffffffll) return CDDT_ERR_ARG;
    // scratch: bucket[n], perm[n], hist[S + 1], cursor[S + 1], scan scratch
    const int64_t nb = h->S + 1;
    int64_t need = 8 * n + 8 * nb + 8 * (scan_scratch_elems(nb) + 2) + 64;
    if (need > h->qscratch_bytes) {
        CDDT_CUDA(cudaStreamSynchronize(st));
        if (h->qscratch) cudaFree(h->qscratch);
        h->qscratch = nullptr;
        h->qscratch_bytes = 0;
        CDDT_CUDA(cudaMalloc(&h->qscratch, (size_t)need));
        h->qscratch_bytes = need;
    }
    char *p = reinterpret_cast<char *>(h->qscratch);
    uint64_t *scan_scratch = reinterpret_cast<uint64_t *>(p);
    p += 8 * (scan_scratch_elems(nb) + 2);
    uint32_t *bucket = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    uint32_t *perm = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    uint32_t *hist = reinterpret_cast<uint32_t *>(p);
    uint32_t *cursor = hist + nb;
    CDDT_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nb, st));
    unsigned blocks = grid_cap(n, threads, 152 * 64);
    bucket_kernel<<<blocks, threads, 0, st>>>(m, pose, n, bucket, hist);
    exclusive_scan_u32(hist, cursor, nb, scan_scratch, scan_scratch + scan_scratch_elems(nb), st);
    place_kernel<<<blocks, threads, 0, st>>>(bucket, n, cursor, perm);
    if (h->u16) calc_range_sorted_kernel<uint16_t><<<blocks, threads, 0, st>>>(m, pose, perm, out, n);
    else calc_range_sorted_kernel<float><<<blocks, threads, 0, st>>>(m, pose, perm, out, n);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// ------------------------------------------------------------ plans

}  // namespace cddt

struct cddt_plan_s {
    int device = 0;
    std::vector<cddt_filter> filters;
    cddt::FilterDev *filters_dev = nullptr;
    cddt::WorkItem *items_dev = nullptr;
    unsigned long long *queue = nullptr;
    int64_t n_items = 0;
    int32_t max_B = 0;
    int32_t tpp = 8, ppi = 256, block = 256;
    int32_t built_ppi = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace cddt {

static cddt_status plan_items(cddt_plan_s *p, cudaStream_t st)
{
    std::vector<WorkItem> items;
    for (size_t f = 0; f < p->filters.size(); ++f) {
        int64_t P = p->filters[f].P;
        for (int64_t s = 0; s < P; s += p->ppi) {
            WorkItem w;
            w.filter = (int32_t)f;
            w.first = s;
            w.count = (int32_t)std::min<int64_t>(p->ppi, P - s);
            items.push_back(w);
        }
    }
    // largest items first: long filters start early, short ones fill the tail
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &b) { return a.count > b.count; });
    if (p->items_dev) cudaFree(p->items_dev);
    p->items_dev = nullptr;
    p->n_items = (int64_t)items.size();
    CDDT_CUDA(cudaMalloc(&p->items_dev, sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    CDDT_CUDA(cudaMemcpyAsync(p->items_dev, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    p->built_ppi = p->ppi;
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    return CDDT_OK;
}

cddt_status plan_create(const cddt_filter *filters, int32_t n, cudaStream_t st, cddt_plan *out)
{
    cddt_plan_s *p = new cddt_plan_s();
    cudaGetDevice(&p->device);
    p->filters.assign(filters, filters + n);
    std::vector<FilterDev> fd(n);
    for (int32_t f = 0; f < n; ++f) {
        const cddt_filter &F = filters[f];
        FilterDev d;
        d.m = F.map->view();
        d.key_u16 = F.map->u16;
        SensorArgs a{};
        a.part = F.particles_dev;
        a.P = F.P;
        a.beam_off = F.beam_off_dev;
        a.obs = F.obs_dev;
        a.B = F.B;
        a.D = F.pair_offset;
        a.bc = make_beam_consts(F.model);
        a.logw = F.logw_dev;
        d.a = a;
        fd[f] = d;
        p->max_B = std::max(p->max_B, F.B);
    }
    cddt_status rc = CDDT_OK;
    cudaError_t e = cudaMalloc(&p->filters_dev, sizeof(FilterDev) * std::max(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->queue, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->filters_dev, fd.data(), sizeof(FilterDev) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc == CDDT_OK) rc = plan_items(p, st);
    if (rc != CDDT_OK) {
        cddt_plan_destroy(p);
        return rc;
    }
    *out = p;
    return CDDT_OK;
}

cddt_status plan_run(cddt_plan_s *p, cudaStream_t st)
{
    if (p->built_ppi != p->ppi) {
        cddt_status rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
    }
    CDDT_CUDA(cudaMemsetAsync(p->queue, 0, sizeof(unsigned long long), st));
    if (p->n_items == 0) return CDDT_OK;
    int blocks_per_sm = 0;
    size_t sm = beam_smem(p->max_B);
    cudaError_t e = cudaSuccess;
    switch (p->tpp) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, batched_kernel<4>, p->block, sm); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, batched_kernel<8>, p->block, sm); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, batched_kernel<16>, p->block, sm); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, batched_kernel<32>, p->block, sm); break;
    }
    CDDT_CUDA(e);
    int nsm = 0;
    CDDT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    int64_t blocks = (int64_t)std::max(blocks_per_sm, 1) * nsm;
    if (blocks > p->n_items) blocks = p->n_items;
    switch (p->tpp) {
    case 4: batched_kernel<4><<<(unsigned)blocks, p->block, sm, st>>>(p->filters_dev, p->items_dev, p->n_items, p->queue, p->max_B); break;
    case 8: batched_kernel<8><<<(unsigned)blocks, p->block, sm, st>>>(p->filters_dev, p->items_dev, p->n_items, p->queue, p->max_B); break;
    case 16: batched_kernel<16><<<(unsigned)blocks, p->block, sm, st>>>(p->filters_dev, p->items_dev, p->n_items, p->queue, p->max_B); break;
    default: batched_kernel<32><<<(unsigned)blocks, p->block, sm, st>>>(p->filters_dev, p->items_dev, p->n_items, p->queue, p->max_B); break;
    }
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

cddt_status plan_launch_graph(cddt_plan_s *p, cudaStream_t st)
{
    if (p->built_ppi != p->ppi) {
        cddt_status rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
    }
    if (!p->exec) {
        cudaStream_t cap;
        CDDT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaStreamDestroy(cap); return cuda_status(e); }
        cddt_status rc = plan_run(p, cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (rc != CDDT_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_status(e);
        p->graph = g;
        CDDT_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
    }
    CDDT_CUDA(cudaGraphLaunch(p->exec, st));
    return CDDT_OK;
}

cddt_status plan_autotune(cddt_plan_s *p, cudaStream_t st)
{
    struct Shape { int tpp, ppi, block; };
    std::vector<Shape> cand;
    for (int tpp : {4, 8, 16, 32})
        for (int block : {128, 256, 512})
            for (int mult : {1, 2, 4, 8}) {
                int ppi = block / tpp * mult;
                cand.push_back({tpp, ppi, block});
            }
    cudaEvent_t e0, e1;
    CDDT_CUDA(cudaEventCreate(&e0));
    CDDT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Shape bs{p->tpp, p->ppi, p->block};
    for (const Shape &s : cand) {
        p->tpp = s.tpp;
        p->ppi = s.ppi;
        p->block = s.block;
        cddt_status rc = plan_run(p, st);  // warm-up (also rebuilds items)
        if (rc != CDDT_OK) continue;
        float tot = 0.f;
        const int reps = 3;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) plan_run(p, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        cudaEventElapsedTime(&tot, e0, e1);
        if (tot < best) { best = tot; bs = s; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tpp = bs.tpp;
    p->ppi = bs.ppi;
    p->block = bs.block;
    return plan_items(p, st);
}

}  // namespace cddt

// C ABI wrappers for plans (the rest of the ABI is in cddt_api.cu).
extern "C" {

cddt_status cddt_plan_create(const cddt_filter *filters_host, int32_t n_filters, void *stream, cddt_plan *out)
{
    if (!filters_host || n_filters <= 0 || !out) return CDDT_ERR_ARG;
    for (int32_t f = 0; f < n_filters; ++f) {
        const cddt_filter &F = filters_host[f];
        if (!F.map || !F.particles_dev || F.P < 0 || !F.beam_off_dev || !F.obs_dev || F.B < 1 ||
            !F.logw_dev || F.model.sigma_hit <= 0 || F.model.max_range <= 0)
            return CDDT_ERR_ARG;
        if (F.pair_offset != 0 && (F.pair_offset >= F.B || 2 * F.pair_offset < F.B)) return CDDT_ERR_ARG;
        if (F.B > 8192) return CDDT_ERR_ARG;
    }
    return cddt::plan_create(filters_host, n_filters, (cudaStream_t)stream, out);
}

cddt_status cddt_plan_autotune(cddt_plan p, void *stream)
{
    if (!p) return CDDT_ERR_ARG;
    return cddt::plan_autotune(p, (cudaStream_t)stream);
}

cddt_status cddt_plan_set_shape(cddt_plan p, int32_t tpp, int32_t ppi, int32_t block)
{
    if (!p) return CDDT_ERR_ARG;
    if (!(tpp == 4 || tpp == 8 || tpp == 16 || tpp == 32)) return CDDT_ERR_ARG;
    if (block < 64 || block > 1024 || block % 32) return CDDT_ERR_ARG;
    if (ppi < 1 || ppi % (32 / tpp)) return CDDT_ERR_ARG;
    p->tpp = tpp;
    p->ppi = ppi;
    p->block = block;
    return CDDT_OK;
}

cddt_status cddt_plan_get_shape(cddt_plan p, int32_t *tpp, int32_t *ppi, int32_t *block)
{
    if (!p) return CDDT_ERR_ARG;
    if (tpp) *tpp = p->tpp;
    if (ppi) *ppi = p->ppi;
    if (block) *block = p->block;
    return CDDT_OK;
}

cddt_status cddt_plan_run(cddt_plan p, void *stream)
{
    if (!p) return CDDT_ERR_ARG;
    return cddt::plan_run(p, (cudaStream_t)stream);
}

cddt_status cddt_plan_launch_graph(cddt_plan p, void *stream)
{
    if (!p) return CDDT_ERR_ARG;
    return cddt::plan_launch_graph(p, (cudaStream_t)stream);
}

int64_t cddt_plan_items(cddt_plan p) { return p ? p->n_items : -1; }

cddt_status cddt_plan_destroy(cddt_plan p)
{
    if (!p) return CDDT_OK;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->filters_dev) cudaFree(p->filters_dev);
    if (p->items_dev) cudaFree(p->items_dev);
    if (p->queue) cudaFree(p->queue);
    delete p;
    return CDDT_OK;
}

}  // extern "C"
