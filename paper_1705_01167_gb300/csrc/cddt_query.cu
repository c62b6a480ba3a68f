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
#include "cddt_sensor.cuh"
#include "cddt_trace.cuh"

namespace cddt {

// ------------------------------------------------------------ single ray

template <typename KT, int SEARCH>
__device__ __forceinline__ Cast cast_one(const MapView &m, float x, float y, float th, uint64_t pol)
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
    cast_pair<KT, SEARCH>(m, x, y, k, false, pol, f, b, kf);
    return kf ? f : b;
}

template <typename KT, int SEARCH>
__global__ void calc_range_kernel(MapView m, const float *pose, float *out, int64_t n)
{
    const uint64_t pol = policy_evict_last();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        float x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        out[q] = cast_one<KT, SEARCH>(m, x, y, th, pol).r;
    }
}

// One query per thread; lane 0 of each warp records the SM cycles from the
// warp's pose loads to its last range store.
template <typename KT, int SEARCH>
__global__ void calc_range_timed_kernel(MapView m, const float *pose, float *out, int64_t n, long long *cycles)
{
    const uint64_t pol = policy_evict_last();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    __syncwarp();
    const long long t0 = clock64();
    if (q < n) {
        const float x = __ldg(pose + 3 * q), y = __ldg(pose + 3 * q + 1), th = __ldg(pose + 3 * q + 2);
        out[q] = cast_one<KT, SEARCH>(m, x, y, th, pol).r;
    }
    __syncwarp();
    const long long t1 = clock64();
    if ((threadIdx.x & 31) == 0 && q < n) cycles[q >> 5] = t1 - t0;
}

cddt_status calc_range_timed(cddt_s *h, const float *pose, float *out, int64_t n, long long *cycles,
                             cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    MapView m = h->view();
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 0x7fffffff) return CDDT_ERR_ARG;
    const bool bin = h->search == CDDT_SEARCH_BINARY;
    if (h->u16 && bin) calc_range_timed_kernel<uint16_t, CDDT_SEARCH_BINARY><<<(unsigned)blocks, threads, 0, st>>>(m, pose, out, n, cycles);
    else if (h->u16) calc_range_timed_kernel<uint16_t, CDDT_SEARCH_TREE><<<(unsigned)blocks, threads, 0, st>>>(m, pose, out, n, cycles);
    else if (bin) calc_range_timed_kernel<float, CDDT_SEARCH_BINARY><<<(unsigned)blocks, threads, 0, st>>>(m, pose, out, n, cycles);
    else calc_range_timed_kernel<float, CDDT_SEARCH_TREE><<<(unsigned)blocks, threads, 0, st>>>(m, pose, out, n, cycles);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// Slice bucket of a query: its stored slice, or S when no search is needed.
__device__ __forceinline__ int slice_bucket(const MapView &m, float x, float y, float th)
{
    if (!free_cell(m.grid, m.W, m.H, x, y)) return m.S;
    int k;
    if (!query_dir(th, m.inv_step, m.N, k)) return m.S;
    return k >= m.S ? k - m.S : k;
}

// Counting sort of queries by slice, in three passes over fixed chunks (one
// chunk per block): per-chunk histograms in shared memory, an exclusive scan
// of the bucket-major (bucket, chunk) counts, then a placement pass that
// writes the permutation and the poses in slice order.
constexpr int kSortThreads = 512;

__global__ void bucket_count_kernel(MapView m, const float *pose, int64_t n, int64_t chunk, uint32_t *bucket,
                                    uint32_t *counts, int nbk)
{
    extern __shared__ uint32_t hist[];
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t q0 = (int64_t)blockIdx.x * chunk, q1 = min(n, q0 + chunk);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int b = slice_bucket(m, __ldg(pose + 3 * q), __ldg(pose + 3 * q + 1), __ldg(pose + 3 * q + 2));
        bucket[q] = (uint32_t)b;
        atomicAdd(hist + b, 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) counts[(int64_t)b * gridDim.x + blockIdx.x] = hist[b];
}

__global__ void place_kernel(const uint32_t *bucket, const float *pose, int64_t n, int64_t chunk,
                             const uint32_t *offsets, int nbk, uint32_t *perm, float *pose_sorted)
{
    extern __shared__ uint32_t cursor[];
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) cursor[b] = offsets[(int64_t)b * gridDim.x + blockIdx.x];
    __syncthreads();
    const int64_t q0 = (int64_t)blockIdx.x * chunk, q1 = min(n, q0 + chunk);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        uint32_t pos = atomicAdd(cursor + bucket[q], 1u);
        perm[pos] = (uint32_t)q;
        pose_sorted[3 * (int64_t)pos] = pose[3 * q];
        pose_sorted[3 * (int64_t)pos + 1] = pose[3 * q + 1];
        pose_sorted[3 * (int64_t)pos + 2] = pose[3 * q + 2];
    }
}

template <typename KT, int SEARCH>
__global__ void calc_range_sorted_kernel(MapView m, const float *pose_sorted, const uint32_t *perm, float *out,
                                         int64_t n)
{
    const uint64_t pol = policy_evict_last();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = pose_sorted[3 * i], y = pose_sorted[3 * i + 1], th = pose_sorted[3 * i + 2];
        out[perm[i]] = cast_one<KT, SEARCH>(m, x, y, th, pol).r;
    }
}

// ------------------------------------------------------------ host

// Threads per particle.  Lanes of a warp that work on different particles of
// one filter read nearby bins of the same slices (coherent gathers), so large
// filters use few lanes per particle; small filters need more lanes to fill
// the GPU (about 300 K resident threads).
static int pick_tpp(int64_t P, int B, int D)
{
    const int T = D > 0 ? D : B;
    int64_t want = (300000 + P - 1) / std::max<int64_t>(P, 1);
    int tpp = 1;
    while (tpp < want && tpp < 32 && tpp * 4 <= T) tpp <<= 1;
    return tpp;
}

cddt_status launch_sensor(const cddt_s *h, const SensorArgs &a, int mode, cudaStream_t st)
{
    const int tpp = pick_tpp(a.P, a.B, a.D);
    if (mode == MODE_FWD && h->search == CDDT_SEARCH_BINARY) return launch_sensor_binary(h, a, tpp, 256, st);
    return h->u16 ? launch_sensor_u16(h, a, mode, tpp, 256, st) : launch_sensor_f32(h, a, mode, tpp, 256, st);
}

cddt_status calc_range(cddt_s *h, const float *pose, float *out, int64_t n, int sorted, cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    MapView m = h->view();
    const int threads = 256;
    if (!sorted) {
        unsigned blocks = grid_cap(n, threads, 152 * 64);
        const bool bin = h->search == CDDT_SEARCH_BINARY;
        if (h->u16 && bin) calc_range_kernel<uint16_t, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose, out, n);
        else if (h->u16) calc_range_kernel<uint16_t, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose, out, n);
        else if (bin) calc_range_kernel<float, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose, out, n);
        else calc_range_kernel<float, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose, out, n);
        CDDT_CUDA(cudaGetLastError());
        return CDDT_OK;
    }
    if (n > 0xffffffffll) return CDDT_ERR_ARG;
    const int nbk = h->S + 1;
    if ((size_t)nbk * sizeof(uint32_t) > 200 * 1024) return CDDT_ERR_ARG;
    int nsm = 0;
    CDDT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    int64_t nblk = std::min<int64_t>((int64_t)nsm * 4, (n + kSortThreads - 1) / kSortThreads);
    const int64_t chunk = (n + nblk - 1) / nblk;
    nblk = (n + chunk - 1) / chunk;
    const int64_t ncount = (int64_t)nbk * nblk;
    // scratch: scan scratch | counts/offsets | bucket[n] | perm[n] | sorted poses[3n]
    int64_t need = 8 * (scan_scratch_elems(ncount) + 2) + 4 * ncount + 4 * n + 4 * n + 12 * n + 256;
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
    p += 8 * (scan_scratch_elems(ncount) + 2);
    uint32_t *counts = reinterpret_cast<uint32_t *>(p);
    p += 4 * ncount;
    p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    uint32_t *bucket = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    uint32_t *perm = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    float *pose_sorted = reinterpret_cast<float *>(p);
    const size_t hs = sizeof(uint32_t) * nbk;
    if (hs > 48 * 1024) {
        CDDT_CUDA(cudaFuncSetAttribute(bucket_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs));
        CDDT_CUDA(cudaFuncSetAttribute(place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs));
    }
    bucket_count_kernel<<<(unsigned)nblk, kSortThreads, hs, st>>>(m, pose, n, chunk, bucket, counts, nbk);
    exclusive_scan_u32(counts, counts, ncount, scan_scratch, scan_scratch + scan_scratch_elems(ncount), st);
    place_kernel<<<(unsigned)nblk, kSortThreads, hs, st>>>(bucket, pose, n, chunk, counts, nbk, perm, pose_sorted);
    unsigned blocks = grid_cap(n, threads, 152 * 64);
    const bool bin = h->search == CDDT_SEARCH_BINARY;
    if (h->u16 && bin) calc_range_sorted_kernel<uint16_t, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else if (h->u16) calc_range_sorted_kernel<uint16_t, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else if (bin) calc_range_sorted_kernel<float, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else calc_range_sorted_kernel<float, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// Slice-sorted ray casting on caller-provided scratch (no allocation).  The
// scratch layout is that of calc_range's sorted path; sorted_scratch_bytes
// gives its size for n queries.
int64_t sorted_scratch_bytes(const cddt_s *h, int64_t n)
{
    const int nbk = h->S + 1;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) return -1;
    int64_t nblk = std::min<int64_t>((int64_t)nsm * 4, (n + kSortThreads - 1) / kSortThreads);
    if (nblk < 1) nblk = 1;
    const int64_t chunk = (n + nblk - 1) / nblk;
    nblk = std::max<int64_t>((n + chunk - 1) / std::max<int64_t>(chunk, 1), 1);
    const int64_t ncount = (int64_t)nbk * nblk;
    return 8 * (scan_scratch_elems(ncount) + 2) + 4 * ncount + 16 + 4 * n + 4 * n + 12 * n;
}

cddt_status calc_range_sorted_into(cddt_s *h, const float *pose, float *out, int64_t n, void *scratch,
                                   int64_t scratch_bytes, cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    MapView m = h->view();
    const int threads = 256;
    const int nbk = h->S + 1;
    const size_t hs = sizeof(uint32_t) * nbk;
    if (hs > 48 * 1024) return CDDT_ERR_ARG;
    int nsm = 0;
    CDDT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    int64_t nblk = std::min<int64_t>((int64_t)nsm * 4, (n + kSortThreads - 1) / kSortThreads);
    const int64_t chunk = (n + nblk - 1) / nblk;
    nblk = (n + chunk - 1) / chunk;
    const int64_t ncount = (int64_t)nbk * nblk;
    if (sorted_scratch_bytes(h, n) > scratch_bytes) return CDDT_ERR_ARG;
    char *p = reinterpret_cast<char *>(scratch);
    uint64_t *scan_scratch = reinterpret_cast<uint64_t *>(p);
    p += 8 * (scan_scratch_elems(ncount) + 2);
    uint32_t *counts = reinterpret_cast<uint32_t *>(p);
    p += 4 * ncount;
    p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    uint32_t *bucket = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    uint32_t *perm = reinterpret_cast<uint32_t *>(p);
    p += 4 * n;
    float *pose_sorted = reinterpret_cast<float *>(p);
    bucket_count_kernel<<<(unsigned)nblk, kSortThreads, hs, st>>>(m, pose, n, chunk, bucket, counts, nbk);
    exclusive_scan_u32(counts, counts, ncount, scan_scratch, scan_scratch + scan_scratch_elems(ncount), st);
    place_kernel<<<(unsigned)nblk, kSortThreads, hs, st>>>(bucket, pose, n, chunk, counts, nbk, perm, pose_sorted);
    const unsigned blocks = grid_cap(n, threads, 152 * 64);
    const bool bin = h->search == CDDT_SEARCH_BINARY;
    if (h->u16 && bin) calc_range_sorted_kernel<uint16_t, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else if (h->u16) calc_range_sorted_kernel<uint16_t, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else if (bin) calc_range_sorted_kernel<float, CDDT_SEARCH_BINARY><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    else calc_range_sorted_kernel<float, CDDT_SEARCH_TREE><<<blocks, threads, 0, st>>>(m, pose_sorted, perm, out, n);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// ------------------------------------------------------------ plans

}  // namespace cddt

struct cddt_plan_s {
    int device = 0;
    std::vector<cddt_filter> filters;
    std::vector<uint64_t> gens;  // handle generations the device descriptors were made from
    cddt::FilterDev *filters_dev = nullptr;
    cddt::WorkItem *items_dev = nullptr;
    unsigned long long *queue = nullptr;
    int64_t n_items = 0;
    int64_t group_start[5] = {0, 0, 0, 0, 0};  // items of (key type, search) group q: [start[q], start[q+1])
    int32_t max_B = 0;
    int32_t tpp = 1, ppi = 512, block = 512, regcap = 0;
    int32_t built_ppi = 0;
    // one launch per (key type, search) group and batch of at most kHotMax
    // filters: its item range and the filters' hot table (a kernel parameter)
    struct Launch {
        int q;
        int64_t first, count;
    };
    std::vector<Launch> launches;
    std::vector<cddt::HotTable> tabs;  // one per launch
    int32_t n_queue = 0;              // queue counters allocated
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace cddt {

static BatchedFn batched_fn(bool u16, int search, int tpp, int block, int regcap)
{
    return u16 ? batched_fn_u16(search, tpp, block, regcap) : batched_fn_f32(search, tpp, block, regcap);
}

static int plan_group_of(const cddt_plan_s *p, size_t f)
{
    const cddt_s *m = p->filters[f].map;
    return (m->u16 ? 2 : 0) + (m->search == CDDT_SEARCH_BINARY ? 1 : 0);
}

// Work items and launches.  Filters are grouped by key type and search
// layout (one kernel instantiation each) and batched kHotMax at a time;
// within a launch the largest items go first: long filters start early,
// short ones fill the tail.  Also rebuilds the hot tables from the handles'
// current views.
static cddt_status plan_items(cddt_plan_s *p, cudaStream_t st)
{
    std::vector<WorkItem> items;
    p->launches.clear();
    p->tabs.clear();
    for (int q = 0; q < 5; ++q) p->group_start[q] = 0;
    for (int q = 0; q < 4; ++q) {
        std::vector<int32_t> fl;
        for (size_t f = 0; f < p->filters.size(); ++f)
            if (p->filters[f].P > 0 && plan_group_of(p, f) == q) fl.push_back((int32_t)f);
        for (size_t b0 = 0; b0 < fl.size(); b0 += kHotMax) {
            const size_t nb = std::min<size_t>(kHotMax, fl.size() - b0);
            HotTable tab;
            std::memset(&tab, 0, sizeof(tab));
            const size_t first = items.size();
            for (size_t i = 0; i < nb; ++i) {
                const cddt_filter &F = p->filters[fl[b0 + i]];
                tab.f[i].m = F.map->view();
                tab.f[i].bc = make_beam_consts(F.model);
                tab.f[i].B = F.B;
                tab.f[i].D = F.pair_offset;
                for (int64_t s0 = 0; s0 < F.P; s0 += p->ppi) {
                    WorkItem w{};
                    w.filter = fl[b0 + i];
                    w.first = s0;
                    w.count = (int32_t)std::min<int64_t>(p->ppi, F.P - s0);
                    w.hot = (int32_t)i;
                    items.push_back(w);
                }
            }
            std::stable_sort(items.begin() + first, items.end(),
                             [](const WorkItem &a, const WorkItem &b) { return a.count > b.count; });
            p->launches.push_back({q, (int64_t)first, (int64_t)(items.size() - first)});
            p->tabs.push_back(tab);
            p->group_start[q + 1] += (int64_t)(items.size() - first);
        }
    }
    for (int q = 0; q < 4; ++q) p->group_start[q + 1] += p->group_start[q];
    if (p->items_dev) cudaFree(p->items_dev);
    p->items_dev = nullptr;
    p->n_items = (int64_t)items.size();
    CDDT_CUDA(cudaMalloc(&p->items_dev, sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    CDDT_CUDA(cudaMemcpyAsync(p->items_dev, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st));
    const int32_t nq = std::max<int32_t>((int32_t)p->launches.size(), 1);
    if (nq > p->n_queue) {
        if (p->queue) cudaFree(p->queue);
        p->queue = nullptr;
        p->n_queue = 0;
        CDDT_CUDA(cudaMalloc(&p->queue, sizeof(unsigned long long) * nq));
        p->n_queue = nq;
    }
    CDDT_CUDA(cudaStreamSynchronize(st));
    p->built_ppi = p->ppi;
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    return CDDT_OK;
}

// Upload the per-filter descriptors (map views are taken from the handles
// now, so a pruned, updated or re-configured handle is seen by later runs).
static cddt_status plan_upload(cddt_plan_s *p, cudaStream_t st)
{
    const int32_t n = (int32_t)p->filters.size();
    std::vector<FilterDev> fd(n);
    p->gens.resize(n);
    for (int32_t f = 0; f < n; ++f) {
        const cddt_filter &F = p->filters[f];
        FilterDev d{};
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
        p->gens[f] = F.map->generation;
    }
    CDDT_CUDA(cudaMemcpyAsync(p->filters_dev, fd.data(), sizeof(FilterDev) * n, cudaMemcpyHostToDevice, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    return CDDT_OK;
}

static bool plan_stale(const cddt_plan_s *p)
{
    for (size_t f = 0; f < p->filters.size(); ++f)
        if (p->filters[f].map->generation != p->gens[f]) return true;
    return false;
}

cddt_status plan_create(const cddt_filter *filters, int32_t n, cudaStream_t st, cddt_plan *out)
{
    cddt_plan_s *p = new cddt_plan_s();
    cudaGetDevice(&p->device);
    p->filters.assign(filters, filters + n);
    for (int32_t f = 0; f < n; ++f) p->max_B = std::max(p->max_B, filters[f].B);
    cddt_status rc = CDDT_OK;
    cudaError_t e = cudaMalloc(&p->filters_dev, sizeof(FilterDev) * std::max(n, 1));
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc == CDDT_OK) rc = plan_upload(p, st);
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
    if (plan_stale(p)) {  // new views, and items regrouped by key type and search layout
        cddt_status rc = plan_upload(p, st);
        if (rc == CDDT_OK) rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
    }
    if (p->built_ppi != p->ppi) {
        cddt_status rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
    }
    CDDT_CUDA(cudaMemsetAsync(p->queue, 0, sizeof(unsigned long long) * p->n_queue, st));
    if (p->n_items == 0) return CDDT_OK;
    size_t sm = beam_smem(p->max_B);
    int nsm = 0;
    CDDT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    for (size_t li = 0; li < p->launches.size(); ++li) {
        const int q = p->launches[li].q;
        const int64_t first = p->launches[li].first;
        const int64_t count = p->launches[li].count;
        if (count == 0) continue;
        const bool u16 = q >= 2;
        const int search = (q & 1) ? CDDT_SEARCH_BINARY : CDDT_SEARCH_TREE;
        BatchedFn fn = batched_fn(u16, search, p->tpp, p->block, p->regcap);
        if (!fn) return CDDT_ERR_ARG;
        if (sm > 48 * 1024) CDDT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int blocks_per_sm = 0;
        CDDT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, p->block, sm));
        int64_t blocks = (int64_t)std::max(blocks_per_sm, 1) * nsm;
        if (blocks > count) blocks = count;
        fn<<<(unsigned)blocks, p->block, sm, st>>>(p->tabs[li], p->filters_dev, p->items_dev + first, count,
                                                   p->queue + li, p->max_B);
    }
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

cddt_status plan_launch_graph(cddt_plan_s *p, cudaStream_t st)
{
    if (plan_stale(p)) {
        cddt_status rc = plan_upload(p, st);
        if (rc == CDDT_OK) rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
    }
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
    struct Shape { int tpp, ppi, block, regcap; };
    std::vector<Shape> cand;
    for (int regcap : {0, 1})
        for (int tpp : {1, 2, 4, 8})
            for (int block : {256, 512})
                for (int mult : {1, 2, 4}) {
                    int ppi = block / tpp * mult;
                    cand.push_back({tpp, ppi, block, regcap});
                }
    cudaEvent_t e0, e1;
    CDDT_CUDA(cudaEventCreate(&e0));
    CDDT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Shape bs{p->tpp, p->ppi, p->block, p->regcap};
    for (const Shape &s : cand) {
        p->tpp = s.tpp;
        p->ppi = s.ppi;
        p->block = s.block;
        p->regcap = s.regcap;
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
    p->regcap = bs.regcap;
    return plan_items(p, st);
}

}  // namespace cddt

// C ABI wrappers for plans (the rest of the ABI is in cddt_api.cu).
extern "C" {

cddt_status cddt_plan_create(const cddt_filter *filters_host, int32_t n_filters, void *stream, cddt_plan *out)
{
    CDDT_RANGE("cddt_plan_create", stream);
    if (!filters_host || n_filters <= 0 || !out) return CDDT_ERR_ARG;
    for (int32_t f = 0; f < n_filters; ++f) {
        const cddt_filter &F = filters_host[f];
        if (!F.map || F.P < 0 || F.B < 1 || !(F.model.sigma_hit > 0) || !(F.model.max_range > 0) ||
            !(F.model.lambda_short > 0))
            return CDDT_ERR_ARG;
        if (F.P > 0 && (!F.particles_dev || !F.beam_off_dev || !F.obs_dev || !F.logw_dev)) return CDDT_ERR_ARG;
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

cddt_status cddt_plan_set_shape(cddt_plan p, int32_t tpp, int32_t ppi, int32_t block, int32_t regcap)
{
    if (!p) return CDDT_ERR_ARG;
    if (!(tpp == 1 || tpp == 2 || tpp == 4 || tpp == 8)) return CDDT_ERR_ARG;
    if (!(block == 256 || block == 512)) return CDDT_ERR_ARG;
    if (ppi < 1 || ppi % (32 / tpp)) return CDDT_ERR_ARG;
    if (regcap != 0 && regcap != 1) return CDDT_ERR_ARG;
    p->tpp = tpp;
    p->ppi = ppi;
    p->block = block;
    p->regcap = regcap;
    return CDDT_OK;
}

cddt_status cddt_plan_get_shape(cddt_plan p, int32_t *tpp, int32_t *ppi, int32_t *block, int32_t *regcap)
{
    if (!p) return CDDT_ERR_ARG;
    if (tpp) *tpp = p->tpp;
    if (ppi) *ppi = p->ppi;
    if (block) *block = p->block;
    if (regcap) *regcap = p->regcap;
    return CDDT_OK;
}

cddt_status cddt_plan_run(cddt_plan p, void *stream)
{
    CDDT_RANGE("cddt_plan_run", stream);
    if (!p) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_plan_run");
    return cddt::plan_run(p, (cudaStream_t)stream);
}

cddt_status cddt_plan_launch_graph(cddt_plan p, void *stream)
{
    CDDT_RANGE("cddt_plan_launch_graph", stream);
    if (!p) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_plan_launch_graph");
    return cddt::plan_launch_graph(p, (cudaStream_t)stream);
}

int64_t cddt_plan_items(cddt_plan p) { return p ? p->n_items : -1; }

cddt_status cddt_plan_groups(cddt_plan p, int64_t *items_per_group)
{
    if (!p || !items_per_group) return CDDT_ERR_ARG;
    for (int q = 0; q < 4; ++q) items_per_group[q] = p->group_start[q + 1] - p->group_start[q];
    return CDDT_OK;
}

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
