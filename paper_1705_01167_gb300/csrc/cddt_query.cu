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
#include <atomic>
#include <cstdlib>
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

// ------------------------------------------------------------ slice-sorted casts
//
// Section IV-C keeps one set of zero points per stored slice.  A batch
// ordered by slice gathers from one slice's bins at a time (a 2000 x 2000
// map's slice holds ~3 MB of its 288 MB store), so the bins a warp reads
// were mostly brought into L2 by the queries just before it.  The order is
// made by a counting sort on the device:
//   count  per block of the batch, its queries of each bucket (a bucket is
//          one direction of one stored slice, or 2^sh consecutive ones when
//          they outnumber kMaxSortBuckets).  The bucket depends on the
//          heading alone, so this pass reads the poses and nothing else;
//   scan   bucket-major exclusive scan of the (bucket, block) counts: the
//          first slot of each block's queries of each bucket;
//   place  each block re-reads its queries a tile at a time, applies the
//          occupancy pre-check, groups the tile by bucket in shared memory
//          and writes one 16-byte record per query, {x, y, query index,
//          slice | flags}, consecutive threads to consecutive slots;
//   cast   one thread per record, in record order: project into the slice
//          (the float32 steps of the unsorted cast), search the bin and
//          write the range to the query's output slot.
// Poses move in 16-byte loads through shared memory (a tile of kSortTile
// poses is 24 KB) whenever the batch starts on a 16-byte boundary.
// Record flags (high bits of its last word, below them the stored slice).
constexpr uint32_t kRecReverse = 0x80000000u;  // search backwards (direction k >= N/2)
constexpr uint32_t kRecZero = 0x40000000u;     // occupied or off-map cell, non-finite pose: range 0
constexpr uint32_t kRecSlice = 0x3fffffffu;

// Sort bucket of a heading: (2 slice + reverse) >> sh, so that the two
// directions of a slice are neighbouring buckets and a warp's records search
// one way (-1 for a non-finite heading, which goes to bucket 0 with a record
// of range 0).
__device__ __forceinline__ int sort_bucket(const MapView &m, float th, int sh, int &s, bool &rev)
{
    int k;
    if (!query_dir(th, m.inv_step, m.N, k)) {
        s = 0;
        rev = false;
        return -1;
    }
    rev = k >= m.S;
    s = rev ? k - m.S : k;
    return ((s << 1) | (rev ? 1 : 0)) >> sh;
}

// Asynchronous copy of 16 bytes from global to shared memory (cp.async,
// completed by cp_async_wait).
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Start copying the poses of queries [t0, t0 + cnt) (cnt <= kSortTile) into
// sp[3 cnt], by the whole block: asynchronous 16-byte copies when the tile
// starts on a 16-byte boundary (its last few floats, and every float of an
// unaligned tile, by plain loads).  Complete after cp_async_wait and a
// barrier.
__device__ __forceinline__ void load_pose_tile(const float *pose, int64_t t0, int cnt, float *sp)
{
    const float *src = pose + 3 * t0;
    const int nf = 3 * cnt;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int n4 = nf >> 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) cp_async16(sp + 4 * i, src + 4 * i);
        done = n4 << 2;
    }
    for (int i = done + threadIdx.x; i < nf; i += blockDim.x) sp[i] = __ldg(src + i);
    cp_async_commit();
}

// Bytes of one tile's poses.
constexpr int kPoseBuf = 3 * (int)sizeof(float) * kSortTile;

__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(MapView m, const float *pose, int64_t n,
                                                                  int64_t chunk, int sh, int nbk, uint32_t *counts)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // pose buffer i & 1 of tile i at smem + (i & 1) * kPoseBuf
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + 2 * kPoseBuf);
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) hist[b] = 0;
    const int64_t q0 = (int64_t)blockIdx.x * chunk, q1 = min(n, q0 + chunk);
    if (q0 < q1) load_pose_tile(pose, q0, (int)min((int64_t)kSortTile, q1 - q0), reinterpret_cast<float *>(smem));
    int it = 0;
    for (int64_t t0 = q0; t0 < q1; t0 += kSortTile, ++it) {
        const int cnt = (int)min((int64_t)kSortTile, q1 - t0);
        const int64_t t1 = t0 + kSortTile;
        if (t1 < q1) {  // the next tile's copies run while this one is counted
            load_pose_tile(pose, t1, (int)min((int64_t)kSortTile, q1 - t1),
                           reinterpret_cast<float *>(smem + ((it + 1) & 1) * kPoseBuf));
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *sp = reinterpret_cast<const float *>(smem + (it & 1) * kPoseBuf);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            int s;
            bool rev;
            const int b = sort_bucket(m, sp[3 * i + 2], sh, s, rev);
            atomicAdd(hist + (b < 0 ? 0 : b), 1u);
        }
        __syncthreads();  // this buffer is free for the tile after next
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) counts[(int64_t)b * gridDim.x + blockIdx.x] = hist[b];
}

__host__ __device__ constexpr size_t count_smem(int nbk)
{
    return 2 * (size_t)kPoseBuf + sizeof(uint32_t) * (size_t)nbk;
}

// Shared memory of sort_place_kernel for nbk buckets: two buffers of
// kSortTile records (tile i's poses land in buffer i & 1 while tile i - 1 is
// placed; its records then overwrite them, grouped by bucket), and per
// bucket the next output slot, the tile's count, its first tile slot and
// the difference of the two (a record at tile slot p goes to output slot
// p + that difference).
constexpr int kRecBuf = kSortTile * (int)sizeof(uint4);
__host__ __device__ constexpr size_t place_smem(int nbk)
{
    return 2 * (size_t)kRecBuf + sizeof(uint32_t) * (4 * (size_t)nbk + 1);
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_place_kernel(MapView m, const float *pose, int64_t n,
                                                                     int64_t chunk, int sh, int nbk,
                                                                     const uint32_t *offsets, uint4 *rec)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // buffer i & 1 at smem + (i & 1) * kRecBuf: tile i's poses, then its records
    uint32_t *cursor = reinterpret_cast<uint32_t *>(smem + 2 * kRecBuf);     // next output slot per bucket
    uint32_t *thist = cursor + nbk;                                          // the tile's queries per bucket
    uint32_t *toff = thist + nbk;                                            // their first tile slot; [nbk] = total
    uint32_t *dbase = toff + nbk + 1;                                        // cursor - toff (mod 2^32)
    for (int b = threadIdx.x; b < nbk; b += blockDim.x) {
        cursor[b] = offsets[(int64_t)b * gridDim.x + blockIdx.x];
        thist[b] = 0;
    }
    const int64_t q0 = (int64_t)blockIdx.x * chunk, q1 = min(n, q0 + chunk);
    if (q0 < q1) load_pose_tile(pose, q0, (int)min((int64_t)kSortTile, q1 - q0), reinterpret_cast<float *>(smem));
    int it = 0;
    for (int64_t t0 = q0; t0 < q1; t0 += kSortTile, ++it) {
        const int cnt = (int)min((int64_t)kSortTile, q1 - t0);
        const int64_t t1 = t0 + kSortTile;
        if (t1 < q1) {  // the next tile's copies run while this one is placed
            load_pose_tile(pose, t1, (int)min((int64_t)kSortTile, q1 - t1),
                           reinterpret_cast<float *>(smem + ((it + 1) & 1) * kRecBuf));
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *sp = reinterpret_cast<const float *>(smem + (it & 1) * kRecBuf);
        uint4 *trec = reinterpret_cast<uint4 *>(smem + (it & 1) * kRecBuf);
        // kSortPerThread queries per thread: buckets and grid cells first,
        // then every grid read, then the projections and the ranks
        // (independent reads in flight together)
        float x[kSortPerThread], y[kSortPerThread];
        int sl[kSortPerThread], bk[kSortPerThread], rank[kSortPerThread];
        int64_t cell[kSortPerThread];
        bool rv[kSortPerThread];
#pragma unroll
        for (int j = 0; j < kSortPerThread; ++j) {
            const int i = j * kSortThreads + threadIdx.x;
            bk[j] = -1;
            cell[j] = -1;
            if (i >= cnt) continue;
            x[j] = sp[3 * i];
            y[j] = sp[3 * i + 1];
            const int b = sort_bucket(m, sp[3 * i + 2], sh, sl[j], rv[j]);
            bk[j] = b < 0 ? 0 : b;
            if (b >= 0) cell[j] = map_cell(m.W, m.H, x[j], y[j]);
        }
        uint8_t occ[kSortPerThread];
#pragma unroll
        for (int j = 0; j < kSortPerThread; ++j) occ[j] = cell[j] >= 0 ? __ldg(m.grid + cell[j]) : 1;
        uint4 r[kSortPerThread];
#pragma unroll
        for (int j = 0; j < kSortPerThread; ++j) {
            rank[j] = 0;
            r[j] = make_uint4(__float_as_uint(x[j]), __float_as_uint(y[j]), (uint32_t)(t0 + j * kSortThreads + threadIdx.x),
                              (uint32_t)sl[j] | (rv[j] ? kRecReverse : 0u) | (occ[j] ? kRecZero : 0u));
        }
#pragma unroll
        for (int j = 0; j < kSortPerThread; ++j)
            if (bk[j] >= 0) rank[j] = (int)atomicAdd(thist + bk[j], 1u);
        __syncthreads();  // the poses are read, the tile's counts complete
        if (threadIdx.x < 32) {  // exclusive scan of the tile's bucket counts
            const int lane = threadIdx.x, per = (nbk + 31) >> 5, b0 = lane * per;
            uint32_t sum = 0;
            for (int i = 0; i < per; ++i)
                if (b0 + i < nbk) sum += thist[b0 + i];
            uint32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            uint32_t run = inc - sum;
            for (int i = 0; i < per; ++i)
                if (b0 + i < nbk) {
                    toff[b0 + i] = run;
                    dbase[b0 + i] = cursor[b0 + i] - run;
                    run += thist[b0 + i];
                }
            if (lane == 31) toff[nbk] = inc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortPerThread; ++j)
            if (bk[j] >= 0) trec[(int)toff[bk[j]] + rank[j]] = r[j];
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint4 v = trec[p];
            // the record's bucket from its slice and direction (a non-finite
            // heading's record has slice 0, forward: bucket 0, as counted)
            const int b = (int)((((v.w & kRecSlice) << 1) | (v.w >> 31)) >> sh);
            rec[(size_t)(dbase[b] + (uint32_t)p)] = v;
        }
        __syncthreads();  // the records are written out: the buffer and the counts are free
        for (int b = threadIdx.x; b < nbk; b += blockDim.x) {
            cursor[b] += thist[b];
            thist[b] = 0;
        }
    }
}

// One thread per record (a stored slice's queries in one direction are
// consecutive records): the unsorted cast's projection, bin and search.
template <typename KT, int SEARCH>
__global__ void __launch_bounds__(256) cast_records_kernel(MapView m, const uint4 *rec, int64_t n, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t pol = policy_evict_normal();
    const uint4 r = __ldcs(rec + i);
    float range = 0.0f;
    if (!(r.w & kRecZero)) {
        const int s = (int)(r.w & kRecSlice);
        float4 sa;
        float X = 0.0f;
        if constexpr (sizeof(KT) == 4) {
            sa = __ldg(chk_slice(m, reinterpret_cast<const float4 *>(m.slices + s), 16));
        } else {  // the whole 32-byte slice record, with the key offset X
            uint32_t w[8];
            ld_node(chk_slice(m, m.slices + s, 32), w);
            sa = make_float4(__uint_as_float(w[0]), __uint_as_float(w[1]), __uint_as_float(w[2]),
                             __uint_as_float(w[3]));
            X = __uint_as_float(w[4]);
        }
        float xr, yr;
        project(__uint_as_float(r.x), __uint_as_float(r.y), sa.x, sa.y, xr, yr);
        const uint32_t Tnb = __float_as_uint(sa.w);
        const int b = query_bin(yr, (int)(Tnb & 0xffffu));
        range = m.max_range;
        if (b >= 0 && b < (int)(Tnb >> 16)) {
            const uint32_t g = __float_as_uint(sa.z) + (uint32_t)b;
            int kb;
            if (!(r.w & kRecReverse)) {  // forward: first key > x'
                const SearchResult sr = bin_search<KT, true, SEARCH>(m, g, xr, X, pol, kb);
                if (sr.idx < kb) {
                    const float d = __fsub_rn(sr.at, xr);
                    if (d < m.max_range) range = d;
                }
            } else {  // reverse: last key < x'
                const SearchResult sr = bin_search<KT, false, SEARCH>(m, g, xr, X, pol, kb);
                if (sr.idx > 0) {
                    const float d = __fsub_rn(xr, sr.prev);
                    if (d < m.max_range) range = d;
                }
            }
        }
    }
    out[r.z] = range;
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

// Shape of the slice sort for n queries.
struct SortShape {
    int sh, nbk;                   // bucket = slice >> sh, nbk buckets
    int64_t nblk, chunk, ncount;   // blocks, queries per block, (bucket, block) counts
};

// Blocks of the count and place passes that fit on one streaming
// multiprocessor at once (both passes use the same blocks).
// Blocks of the count and place passes that fit on one streaming
// multiprocessor at once, for the largest bucket count (the shared memory of
// both passes grows with it), queried once per device; the first query also
// raises both kernels' shared-memory limits.  0 when a query failed.
static int sort_blocks_per_sm()
{
    constexpr int kDevices = 64;
    static std::atomic<int> cached[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < kDevices) {
        const int v = cached[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int a = 0, b = 0;
    if (cudaFuncSetAttribute(sort_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)count_smem(kMaxSortBuckets)) != cudaSuccess ||
        cudaFuncSetAttribute(sort_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)place_smem(kMaxSortBuckets)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, sort_count_kernel, kSortThreads,
                                                      count_smem(kMaxSortBuckets)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sort_place_kernel, kSortThreads,
                                                      place_smem(kMaxSortBuckets)) != cudaSuccess)
        return 0;
    const int v = std::max(1, std::min(a, b));
    if (dev < kDevices) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

static SortShape sort_shape(const cddt_s *h, int64_t n)
{
    SortShape p;
    p.sh = 0;
    while (((2 * h->S - 1) >> p.sh) + 1 > kMaxSortBuckets) ++p.sh;
    p.nbk = ((2 * h->S - 1) >> p.sh) + 1;
    // one wave of blocks, each a whole number of tiles
    const int64_t nn = std::max<int64_t>(n, 1);
    const int64_t waves = (int64_t)sm_count() * std::max(1, sort_blocks_per_sm());
    const int64_t tiles = (nn + kSortTile - 1) / kSortTile;
    p.chunk = ((tiles + waves - 1) / waves) * kSortTile;
    p.nblk = (nn + p.chunk - 1) / p.chunk;
    p.ncount = (int64_t)p.nbk * p.nblk;
    return p;
}

// Scratch of the sort: scan partials and total | (bucket, block) counts |
// 16-byte aligned records, one per query.
static int64_t sort_scratch_bytes(const SortShape &p, int64_t n)
{
    return 8 * (scan_scratch_elems(p.ncount) + 2) + 4 * p.ncount + 16 + 16 * n;
}

int64_t sorted_scratch_bytes(const cddt_s *h, int64_t n) { return sort_scratch_bytes(sort_shape(h, n), n); }

cddt_status calc_range_sorted_into(cddt_s *h, const float *pose, float *out, int64_t n, void *scratch,
                                   int64_t scratch_bytes, cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    if (n > 0xffffffffll) return CDDT_ERR_ARG;
    const SortShape p = sort_shape(h, n);
    if (sort_scratch_bytes(p, n) > scratch_bytes) return CDDT_ERR_ARG;
    char *c = reinterpret_cast<char *>(scratch);
    uint64_t *scan_part = reinterpret_cast<uint64_t *>(c);
    uint64_t *total = scan_part + scan_scratch_elems(p.ncount);
    c += 8 * (scan_scratch_elems(p.ncount) + 2);
    uint32_t *counts = reinterpret_cast<uint32_t *>(c);
    c += 4 * p.ncount;
    uint4 *rec = reinterpret_cast<uint4 *>(((uintptr_t)c + 15) & ~(uintptr_t)15);
    const MapView m = h->view();
    if (sort_blocks_per_sm() == 0) return CDDT_ERR_CUDA;  // also raises the kernels' shared-memory limits
    sort_count_kernel<<<(unsigned)p.nblk, kSortThreads, count_smem(p.nbk), st>>>(m, pose, n, p.chunk, p.sh, p.nbk,
                                                                                 counts);
    exclusive_scan_u32(counts, counts, p.ncount, scan_part, total, st);
    sort_place_kernel<<<(unsigned)p.nblk, kSortThreads, place_smem(p.nbk), st>>>(m, pose, n, p.chunk, p.sh, p.nbk,
                                                                                 counts, rec);
    const bool bin = h->search == CDDT_SEARCH_BINARY;
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffff) return CDDT_ERR_ARG;
    const unsigned g = (unsigned)blocks;
    if (h->u16 && bin) cast_records_kernel<uint16_t, CDDT_SEARCH_BINARY><<<g, 256, 0, st>>>(m, rec, n, out);
    else if (h->u16) cast_records_kernel<uint16_t, CDDT_SEARCH_TREE><<<g, 256, 0, st>>>(m, rec, n, out);
    else if (bin) cast_records_kernel<float, CDDT_SEARCH_BINARY><<<g, 256, 0, st>>>(m, rec, n, out);
    else cast_records_kernel<float, CDDT_SEARCH_TREE><<<g, 256, 0, st>>>(m, rec, n, out);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

cddt_status calc_range(cddt_s *h, const float *pose, float *out, int64_t n, int sorted, cudaStream_t st)
{
    if (n == 0) return CDDT_OK;
    if (!sorted) {
        const MapView m = h->view();
        const unsigned blocks = grid_cap(n, 256, 64);
        const bool bin = h->search == CDDT_SEARCH_BINARY;
        if (h->u16 && bin) calc_range_kernel<uint16_t, CDDT_SEARCH_BINARY><<<blocks, 256, 0, st>>>(m, pose, out, n);
        else if (h->u16) calc_range_kernel<uint16_t, CDDT_SEARCH_TREE><<<blocks, 256, 0, st>>>(m, pose, out, n);
        else if (bin) calc_range_kernel<float, CDDT_SEARCH_BINARY><<<blocks, 256, 0, st>>>(m, pose, out, n);
        else calc_range_kernel<float, CDDT_SEARCH_TREE><<<blocks, 256, 0, st>>>(m, pose, out, n);
        CDDT_CUDA(cudaGetLastError());
        return CDDT_OK;
    }
    if (n > 0xffffffffll) return CDDT_ERR_ARG;
    const int64_t need = sorted_scratch_bytes(h, n);
    if (need > h->qscratch_bytes) {
        CDDT_CUDA(cudaStreamSynchronize(st));
        if (h->qscratch) cudaFree(h->qscratch);
        h->qscratch = nullptr;
        h->qscratch_bytes = 0;
        CDDT_CUDA(cudaMalloc(&h->qscratch, (size_t)need));
        h->qscratch_bytes = need;
    }
    return calc_range_sorted_into(h, pose, out, n, h->qscratch, h->qscratch_bytes, st);
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
    std::vector<std::vector<int32_t>> launch_filters;  // per launch, its filters in hot-table order
    int32_t n_queue = 0;              // queue counters allocated
    // gradient refinement (cddt_plan_refine): its own items, blockDim / tpp
    // particles each, per forward launch
    cddt::WorkItem *refine_items_dev = nullptr;
    int32_t refine_tpp = 0;
    std::vector<Launch> refine_launches;
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
    p->launch_filters.clear();
    p->refine_tpp = 0;  // the refinement items follow the launches
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
            p->launch_filters.emplace_back(fl.begin() + b0, fl.begin() + b0 + nb);
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
        a.grad_xy = F.grad_xy_dev;
        a.part_out = F.particles_out_dev;
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

// Refinement items: the filters of every forward launch, cut into items of
// kRefineBlock / tpp particles (one block's particles at once).
static cddt_status refine_items(cddt_plan_s *p, int tpp, cudaStream_t st)
{
    std::vector<WorkItem> items;
    p->refine_launches.clear();
    const int per = kRefineBlock / tpp;
    for (size_t li = 0; li < p->launches.size(); ++li) {
        const size_t first = items.size();
        const std::vector<int32_t> &fl = p->launch_filters[li];
        for (size_t hot = 0; hot < fl.size(); ++hot) {
            const int64_t P = p->filters[fl[hot]].P;
            for (int64_t s0 = 0; s0 < P; s0 += per) {
                WorkItem w{};
                w.filter = fl[hot];
                w.first = s0;
                w.count = (int32_t)std::min<int64_t>(per, P - s0);
                w.hot = (int32_t)hot;
                items.push_back(w);
            }
        }
        p->refine_launches.push_back({p->launches[li].q, (int64_t)first, (int64_t)(items.size() - first)});
    }
    if (p->refine_items_dev) cudaFree(p->refine_items_dev);
    p->refine_items_dev = nullptr;
    CDDT_CUDA(cudaMalloc(&p->refine_items_dev, sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    CDDT_CUDA(cudaMemcpyAsync(p->refine_items_dev, items.data(), sizeof(WorkItem) * items.size(),
                              cudaMemcpyHostToDevice, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    p->refine_tpp = tpp;
    return CDDT_OK;
}

cddt_status plan_refine(cddt_plan_s *p, int32_t steps, float eta, int32_t tpp, cudaStream_t st)
{
    bool rebuilt = false;
    if (plan_stale(p)) {
        cddt_status rc = plan_upload(p, st);
        if (rc == CDDT_OK) rc = plan_items(p, st);
        if (rc != CDDT_OK) return rc;
        rebuilt = true;
    }
    if (tpp == 0) {  // lanes per particle: two waves of resident threads (2048 per SM)
        int64_t total = 0;
        for (const cddt_filter &F : p->filters) total += std::max<int64_t>(F.P, 0);
        const int64_t want = ((int64_t)sm_count() * 4096 + std::max<int64_t>(total, 1) - 1) / std::max<int64_t>(total, 1);
        tpp = 1;
        while (tpp < want && tpp < kRefineBlock) tpp <<= 1;
    }
    if (rebuilt || p->refine_tpp != tpp || !p->refine_items_dev) {
        cddt_status rc = refine_items(p, tpp, st);
        if (rc != CDDT_OK) return rc;
    }
    CDDT_CUDA(cudaMemsetAsync(p->queue, 0, sizeof(unsigned long long) * p->n_queue, st));
    RefineFn fn0 = refine_fn(false, tpp), fn1 = refine_fn(true, tpp);
    if (!fn0 || !fn1) return CDDT_ERR_ARG;
    const size_t sm = beam_smem(p->max_B);
    for (size_t li = 0; li < p->refine_launches.size(); ++li) {
        const int64_t first = p->refine_launches[li].first, count = p->refine_launches[li].count;
        if (count == 0) continue;
        RefineFn fn = p->refine_launches[li].q >= 2 ? fn1 : fn0;
        if (sm > 48 * 1024) CDDT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int blocks_per_sm = 0;
        CDDT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, kRefineBlock, sm));
        int64_t blocks = (int64_t)std::max(blocks_per_sm, 1) * sm_count();
        if (blocks > count) blocks = count;
        fn<<<(unsigned)blocks, kRefineBlock, sm, st>>>(p->tabs[li], p->filters_dev, p->refine_items_dev + first,
                                                        count, p->queue + li, steps, eta);
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
        for (int tpp : {1, 2, 4, 8, 16, 32})
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
    if (!(tpp == 1 || tpp == 2 || tpp == 4 || tpp == 8 || tpp == 16 || tpp == 32)) return CDDT_ERR_ARG;
    if (!(block == 256 || block == 512)) return CDDT_ERR_ARG;
    if (ppi < 1 || ppi % (32 / tpp)) return CDDT_ERR_ARG;
    if (regcap != 0 && regcap != 1) return CDDT_ERR_ARG;
    if (tpp != p->tpp || ppi != p->ppi || block != p->block || regcap != p->regcap) {
        // a graph captured with the old shape would go on launching it
        if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
        if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    }
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

cddt_status cddt_plan_refine(cddt_plan p, int32_t steps, float eta, int32_t tpp, void *stream)
{
    CDDT_RANGE("cddt_plan_refine", stream);
    if (!p) return CDDT_ERR_ARG;
    if (steps < 0 || !(eta >= 0.0f) || !(eta < 1e30f)) return CDDT_ERR_ARG;
    if (!(tpp == 0 || tpp == 1 || tpp == 2 || tpp == 4 || tpp == 8 || tpp == 16 || tpp == 32 || tpp == 64 ||
          tpp == 128 || tpp == 256))
        return CDDT_ERR_ARG;
    for (const cddt_filter &F : p->filters)
        if (F.P > 0 && (!F.grad_xy_dev || !F.particles_out_dev)) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_plan_refine");
    return cddt::plan_refine(p, steps, eta, tpp, (cudaStream_t)stream);
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
    if (p->refine_items_dev) cudaFree(p->refine_items_dev);
    if (p->queue) cudaFree(p->queue);
    delete p;
    return CDDT_OK;
}

}  // extern "C"
