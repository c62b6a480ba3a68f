// cddt_build.cu -- GPU construction of the CDDT (Section IV-A), shared
// scan / sort / index kernels (also used by prune and update).
//
// Construction, following the direct construction algorithm: the edge map
// (occupied cells with a free or off-map 8-neighbour) is computed, every
// (edge cell, slice) pair is projected into the slice and counted in each
// bin its rotated square overlaps, the per-bin counts are laid out into
// 32-byte aligned runs, the projected abscissae are scattered, each bin is
// sorted (the sorted-vector successor structure of Section IV-B) and the
// implicit search tree of every bin is filled from its sorted keys.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

cddt_status cuda_status(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return CDDT_ERR_OOM;
    return CDDT_ERR_CUDA;
}

int sm_count()
{
    constexpr int kDevices = 64;
    static std::atomic<int> cached[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev >= kDevices) {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0 ? v : 1;
    }
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

// ------------------------------------------------------------ scan

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *warp_sums, uint64_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    uint64_t before = wid ? warp_sums[wid - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void scan_reduce_kernel(const uint32_t *in, int64_t n, uint64_t *partial)
{
    __shared__ uint64_t ws[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    uint64_t tot;
    block_exclusive_scan(s, ws, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void scan_partials_kernel(uint64_t *partial, int64_t nblocks, uint64_t *total)
{
    __shared__ uint64_t ws[32];
    uint64_t carry = 0;
    for (int64_t b0 = 0; b0 < nblocks; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        uint64_t v = i < nblocks ? partial[i] : 0;
        uint64_t tot;
        uint64_t ex = block_exclusive_scan(v, ws, tot);
        if (i < nblocks) partial[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_apply_kernel(const uint32_t *in, int64_t n, const uint64_t *partial, uint32_t *out)
{
    __shared__ uint64_t ws[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    uint64_t tot;
    uint64_t ex = block_exclusive_scan(s, ws, tot) + partial[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = (uint32_t)ex;
        ex += v[i];
    }
}

// Exclusive scan of n uint32 values into out (may alias in); the total is
// written to total_dev.  scratch: >= (n / kScanTile + 1) uint64.
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *scratch,
                        uint64_t *total_dev, cudaStream_t st)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), st);
        return;
    }
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, scratch);
    scan_partials_kernel<<<1, 1024, 0, st>>>(scratch, nb, total_dev);
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, scratch, out);
}

int64_t scan_scratch_elems(int64_t n) { return n / kScanTile + 2; }

// ------------------------------------------------------------ grid kernels

__global__ void normalise_grid_kernel(const uint8_t *in, uint8_t *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] ? 1 : 0;
}

// Edge map (Section IV-A: map minus its 3x3 erosion; off-map is free).
__global__ void edge_map_kernel(const uint8_t *g, uint8_t *edge, int W, int H)
{
    int64_t n = (int64_t)W * H;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(q / W), i = (int)(q - (int64_t)j * W);
        edge[q] = edge_at(g, W, H, i, j);
    }
}


// Row-major compaction of nonzero flags into cell indices (deterministic).
__global__ void flag_count_kernel(const uint8_t *flag, int64_t n, uint32_t *block_count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (i < n) && flag[i];
    int c = __syncthreads_count(v);
    if (threadIdx.x == 0) block_count[blockIdx.x] = (uint32_t)c;
}

__global__ void flag_write_kernel(const uint8_t *flag, int64_t n, const uint32_t *block_off, uint32_t *out)
{
    __shared__ uint32_t wcount[32];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (i < n) && flag[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, v);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += wcount[w];
    if (v) out[block_off[blockIdx.x] + before + __popc(m & ((1u << lane) - 1))] = (uint32_t)i;
}

// ------------------------------------------------------------ construction

// Count: every (edge cell, slice) adds one to each bin it overlaps.
__global__ void count_kernel(const uint32_t *cells, int64_t E, int W, const SliceInfo *slices, int S,
                             uint32_t *count)
{
    int64_t total = E * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int s = (int)(t / E);
        int64_t e = t - (int64_t)s * E;
        uint32_t q = cells[e];
        int j = (int)(q / (uint32_t)W), i = (int)(q - (uint32_t)j * W);
        SliceInfo si = slices[s];
        float xr, yr;
        project((float)i, (float)j, si.c, si.s, xr, yr);
        int b0, b1;
        if (!cell_bins(yr, half_extent(si.c, si.s), si.T, si.nb, b0, b1)) continue;
        for (int b = b0; b <= b1; ++b) atomicAdd(count + si.sbase + b, 1u);
    }
}

template <int LK, int R>
__global__ void nodes_kernel(const uint32_t *count, int64_t nbins, uint32_t *nodes)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nbins;
         g += (int64_t)gridDim.x * blockDim.x)
        nodes[g] = bin_nodes(count[g], LK, R);
}

__global__ void hdr_kernel(const uint32_t *count, const uint32_t *node_off, int64_t nbins, BinHdr *hdr,
                           unsigned long long *max_bin)
{
    // whole warps step together (blockDim is a multiple of 32), so the
    // warp's largest count takes one atomic
    const int lane = threadIdx.x & 31;
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); g0 < nbins;
         g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + lane;
        unsigned m = 0;
        if (g < nbins) {
            BinHdr b;
            b.off = node_off[g];
            b.nm = count[g];
            for (int q = 0; q < 6; ++q) b.w[q] = 0;
            hdr[g] = b;
            m = b.nm;
        }
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m) atomicMax(max_bin, (unsigned long long)m);
    }
}

// Scatter: the projected abscissa of every (edge cell, slice, bin) into the
// bin's leaf run, at a slot taken from a per-bin cursor (the order is fixed by
// the sort that follows).
template <typename KT>
__global__ void scatter_kernel(const uint32_t *cells, int64_t E, int W, const SliceInfo *slices, int S,
                               const BinHdr *hdr, uint32_t *cursor, void *store, float Q)
{
    int64_t total = E * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int s = (int)(t / E);
        int64_t e = t - (int64_t)s * E;
        uint32_t q = cells[e];
        int j = (int)(q / (uint32_t)W), i = (int)(q - (uint32_t)j * W);
        SliceInfo si = slices[s];
        float xr, yr;
        project((float)i, (float)j, si.c, si.s, xr, yr);
        int b0, b1;
        if (!cell_bins(yr, half_extent(si.c, si.s), si.T, si.nb, b0, b1)) continue;
        for (int b = b0; b <= b1; ++b) {
            uint32_t g = si.sbase + b;
            uint32_t pos = atomicAdd(cursor + g, 1u);
            KT *run = leaf_run<KT>(store, hdr[g].off, bin_count(hdr[g].nm));
            if (sizeof(KT) == 4)
                reinterpret_cast<float *>(run)[pos] = xr;
            else
                reinterpret_cast<uint16_t *>(run)[pos] = quantise(xr, si.X, Q);
        }
    }
}

static unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > (int64_t)sm_count() * 64) b = (int64_t)sm_count() * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}


// ------------------------------------------------------------ segmented sort


// Size classes of the segmented sort: one lane per key, one warp with up to
// 32 keys per lane in registers, a block with 16 keys per thread in registers
// (two sizes), and global memory above.
constexpr uint32_t kWarpSortMax = 32;
constexpr uint32_t kRegSortMax = 1024;
constexpr uint32_t kBlockSortMax = 2048;
constexpr uint32_t kBigSortMax = 16384;
constexpr int kSortClasses = 5;

template <typename KT>
__global__ void classify_kernel(Segs<KT> sg, int64_t nseg, uint32_t *lists, uint32_t *list_n, int64_t cap)
{
    // whole warps step together (blockDim is a multiple of 32): one atomic
    // per warp and size class
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); g0 < nseg;
         g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + lane;
        int cls = -1;  // segments of 0 or 1 keys are sorted already
        if (g < nseg) {
            KT *p;
            uint32_t n;
            sg.get((uint32_t)g, p, n);
            const bool skip = sg.skip_upto && n <= sg.skip_upto &&
                              (!sg.also_len || sg.also_len[g] <= sg.skip_upto);
            if (n <= 1 || skip) cls = -1;
            else if (n <= kWarpSortMax) cls = 0;
            else if (n <= kRegSortMax) cls = 4;
            else if (n <= kBlockSortMax) cls = 1;
            else if (n <= kBigSortMax) cls = 2;
            else cls = 3;
        }
        for (int c = 0; c < kSortClasses; ++c) {
            const unsigned mine = __ballot_sync(0xffffffffu, cls == c);
            if (!mine) continue;
            uint32_t base = 0;
            if (lane == __ffs(mine) - 1) base = atomicAdd(list_n + c, (unsigned)__popc(mine));
            base = __shfl_sync(0xffffffffu, base, __ffs(mine) - 1);
            if (cls == c) lists[c * cap + base + __popc(mine & lt)] = (uint32_t)g;
        }
    }
}

__device__ __forceinline__ float shfl_xor_key(float v, int j) { return __shfl_xor_sync(0xffffffffu, v, j); }
__device__ __forceinline__ uint16_t shfl_xor_key(uint16_t v, int j)
{
    return (uint16_t)__shfl_xor_sync(0xffffffffu, (uint32_t)v, j);
}

// Ascending bitonic sort of 32 keys held one per lane.
template <typename KT>
__device__ __forceinline__ KT warp_bitonic(KT v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            KT o = shfl_xor_key(v, j);
            bool up = ((lane & k) == 0);
            bool lower = ((lane & j) == 0);
            KT mn = v < o ? v : o, mx = v < o ? o : v;
            v = (lower == up) ? mn : mx;
        }
    }
    return v;
}

template <typename KT>
__global__ void warp_sort_kernel(Segs<KT> sg, const uint32_t *list, uint32_t count)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count;
         w += (gridDim.x * blockDim.x) >> 5) {
        KT *run;
        uint32_t n;
        sg.get(list[w], run, n);
        KT v = lane < (int)n ? run[lane] : pad_key<KT>();
        v = warp_bitonic<KT>(v);
        if (lane < (int)n) run[lane] = v;
    }
}

// Ascending bitonic sort of 32 M keys held by one warp, M per lane: key
// index i = e * 32 + lane.  Partners at distance >= 32 are in the same lane
// (registers), nearer ones one shuffle away; no barriers.
template <typename KT, int M>
__device__ __forceinline__ void warp_reg_sort(KT *run, int n, int lane)
{
    constexpr int N = 32 * M;
    KT r[M];
#pragma unroll
    for (int e = 0; e < M; ++e) {
        const int i = e * 32 + lane;
        r[e] = i < n ? run[i] : pad_key<KT>();
    }
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int e = 0; e < M; ++e) {
                    const int pe = e ^ (j >> 5);
                    if (pe > e) {
                        const bool up = (((e * 32 + lane) & k) == 0);
                        const KT a = r[e], b = r[pe];
                        const bool sw = up ? (b < a) : (a < b);
                        r[e] = sw ? b : a;
                        r[pe] = sw ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < M; ++e) {
                    const KT o = shfl_xor_key(r[e], j);
                    const bool up = (((e * 32 + lane) & k) == 0);
                    const bool lower = ((lane & j) == 0);
                    const KT mn = r[e] < o ? r[e] : o, mx = r[e] < o ? o : r[e];
                    r[e] = (lower == up) ? mn : mx;
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < M; ++e) {
        const int i = e * 32 + lane;
        if (i < n) run[i] = r[e];
    }
}

// Segments of 33..1024 keys: one warp each, the register width picked per
// segment (warp-uniform).
template <typename KT>
__global__ void reg_sort_kernel(Segs<KT> sg, const uint32_t *list, uint32_t count)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count;
         w += (gridDim.x * blockDim.x) >> 5) {
        KT *run;
        uint32_t n;
        sg.get(list[w], run, n);
        if (n <= 64) warp_reg_sort<KT, 2>(run, (int)n, lane);
        else if (n <= 128) warp_reg_sort<KT, 4>(run, (int)n, lane);
        else if (n <= 256) warp_reg_sort<KT, 8>(run, (int)n, lane);
        else if (n <= 512) warp_reg_sort<KT, 16>(run, (int)n, lane);
        else warp_reg_sort<KT, 32>(run, (int)n, lane);
    }
}

// One register stage of distance J < 16 (keys i = t * 16 + e).
template <typename KT, int J>
__device__ __forceinline__ void reg_stage(KT (&r)[16], uint32_t t, uint32_t k)
{
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int pe = e ^ J;
        if (pe > e) {
            const bool up = ((t * 16 + e) & k) == 0;
            const KT a = r[e], b = r[pe];
            const bool sw = up ? (b < a) : (a < b);
            r[e] = sw ? b : a;
            r[pe] = sw ? a : b;
        }
    }
}

// Segments of 1025..16384 keys: the bitonic network over a power-of-two
// padded copy with thread t holding keys t * 16 .. t * 16 + 15 in registers.
// Distances below 16 are register swaps, 16..256 one shuffle, and only the
// stages of distance >= 512 (across warps) go through shared memory: 15 of
// the 105 stages for 16384 keys.  Threads past the padded size work on pads
// among themselves (i ^ j stays above the size).
template <typename KT, int THREADS>
__global__ void __launch_bounds__(THREADS) block_reg_sort_kernel(Segs<KT> sg, const uint32_t *list, uint32_t count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KT *sh = reinterpret_cast<KT *>(smem_raw);
    const uint32_t t = threadIdx.x;
    const int lane = (int)(t & 31);
    for (uint32_t w = blockIdx.x; w < count; w += gridDim.x) {
        KT *run;
        uint32_t n;
        sg.get(list[w], run, n);
        uint32_t P = 512;
        while (P < n) P <<= 1;
        const bool act = t * 16 < P;  // whole warps: P is a multiple of 512
        KT r[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const uint32_t i = t * 16 + e;
            r[e] = i < n ? run[i] : pad_key<KT>();
        }
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                if (j >= 512) {
                    if (act) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) sh[t * 16 + e] = r[e];
                    }
                    __syncthreads();
                    if (act) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const uint32_t i = t * 16 + e;
                            const KT o = sh[i ^ j];
                            const bool up = (i & k) == 0, lower = (i & j) == 0;
                            const KT mn = r[e] < o ? r[e] : o, mx = r[e] < o ? o : r[e];
                            r[e] = (lower == up) ? mn : mx;
                        }
                    }
                    __syncthreads();
                } else if (!act) {
                    // past the padded size: nothing to do between barriers
                } else if (j >= 16) {
                    const int d = (int)(j >> 4);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const uint32_t i = t * 16 + e;
                        const KT o = shfl_xor_key(r[e], d);
                        const bool up = (i & k) == 0, lower = (lane & d) == 0;
                        const KT mn = r[e] < o ? r[e] : o, mx = r[e] < o ? o : r[e];
                        r[e] = (lower == up) ? mn : mx;
                    }
                } else if (j == 8) {
                    reg_stage<KT, 8>(r, t, k);
                } else if (j == 4) {
                    reg_stage<KT, 4>(r, t, k);
                } else if (j == 2) {
                    reg_stage<KT, 2>(r, t, k);
                } else {
                    reg_stage<KT, 1>(r, t, k);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const uint32_t i = t * 16 + e;
            if (i < n) run[i] = r[e];
        }
    }
}

// Segments larger than shared memory: the same network on a power-of-two
// scratch copy in global memory, one segment at a time.
template <typename KT>
__global__ void global_sort_stage_kernel(KT *buf, uint32_t P, uint32_t k, uint32_t j)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        uint32_t p = i ^ j;
        if (p > i) {
            KT a = buf[i], b = buf[p];
            bool up = (i & k) == 0;
            if ((a > b) == up) { buf[i] = b; buf[p] = a; }
        }
    }
}

template <typename KT>
__global__ void seg_info_kernel(Segs<KT> sg, const uint32_t *list, uint32_t count, unsigned long long *ptr,
                                uint32_t *len)
{
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < count; w += gridDim.x * blockDim.x) {
        KT *p;
        uint32_t n;
        sg.get(list[w], p, n);
        ptr[w] = (unsigned long long)(uintptr_t)p;
        len[w] = n;
    }
}

template <typename KT>
__global__ void copy_pad_kernel(const KT *src, uint32_t n, KT *dst, uint32_t P)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
        dst[i] = i < n ? src[i] : pad_key<KT>();
}

template <typename KT>
__global__ void copy_back_kernel(const KT *src, uint32_t n, KT *dst)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// Pad every bin's last leaf with +inf and fill its tree: the separator of
// child j at level l-1 of a level-l node is the largest key of the child's
// subtree, key[min((j+1) K^l, n) - 1], or +inf past the end; the header holds
// the root's separators over the top stored level, or the keys themselves
// when the bin has at most R keys.
template <typename KT>
__global__ void index_kernel(void *store, BinHdr *hdr, int64_t nbins)
{
    const int lane = threadIdx.x & 31;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5)
        index_bin<KT>(store, hdr, g, lane);
}

// ------------------------------------------------------------ host

// Sort every segment ascending, by size class.  Synchronises `st`.
template <typename KT>
cddt_status sort_segments(const Segs<KT> &sg, int64_t nseg, cudaStream_t st, Arena *ws)
{
    if (nseg == 0) return CDDT_OK;
    Buf lists_b, list_n_b;
    uint32_t *L = ws ? ws->take<uint32_t>(kSortClasses * (size_t)nseg) : nullptr;
    uint32_t *LN = ws ? ws->take<uint32_t>(kSortClasses) : nullptr;
    if (!L || !LN) {
        CDDT_CUDA(lists_b.alloc(sizeof(uint32_t) * kSortClasses * (size_t)nseg));
        CDDT_CUDA(list_n_b.alloc(sizeof(uint32_t) * kSortClasses));
        L = lists_b.as<uint32_t>();
        LN = list_n_b.as<uint32_t>();
    }
    CDDT_CUDA(cudaMemsetAsync(LN, 0, sizeof(uint32_t) * kSortClasses, st));
    classify_kernel<KT><<<grid_for(nseg, 256), 256, 0, st>>>(sg, nseg, L, LN, nseg);
    uint32_t cnt[kSortClasses];
    CDDT_CUDA(cudaMemcpyAsync(cnt, LN, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    if (cnt[4]) reg_sort_kernel<KT><<<grid_for((int64_t)cnt[4] * 32, 256), 256, 0, st>>>(sg, L + 4 * nseg, cnt[4]);
    if (cnt[0]) warp_sort_kernel<KT><<<grid_for((int64_t)cnt[0] * 32, 256), 256, 0, st>>>(sg, L, cnt[0]);
    if (cnt[1]) {  // 1025..2048 keys: 128 threads x 16 keys
        const size_t sm = sizeof(KT) * kBlockSortMax;
        block_reg_sort_kernel<KT, kBlockSortMax / 16><<<std::min<uint32_t>(cnt[1], (uint32_t)sm_count() * 16), kBlockSortMax / 16, sm, st>>>(
            sg, L + nseg, cnt[1]);
    }
    if (cnt[2]) {  // 2049..16384 keys: 1024 threads x 16 keys
        const size_t sm = sizeof(KT) * kBigSortMax;
        CDDT_CUDA(cudaFuncSetAttribute(block_reg_sort_kernel<KT, kBigSortMax / 16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        block_reg_sort_kernel<KT, kBigSortMax / 16><<<std::min<uint32_t>(cnt[2], (uint32_t)sm_count() * 2), kBigSortMax / 16, sm, st>>>(
            sg, L + 2 * nseg, cnt[2]);
    }
    if (cnt[3]) {
        Buf dptr, dlen;
        CDDT_CUDA(dptr.alloc(sizeof(unsigned long long) * cnt[3]));
        CDDT_CUDA(dlen.alloc(sizeof(uint32_t) * cnt[3]));
        seg_info_kernel<KT><<<grid_for(cnt[3], 256), 256, 0, st>>>(sg, L + 3 * nseg, cnt[3], dptr.as<unsigned long long>(), dlen.as<uint32_t>());
        std::vector<unsigned long long> ptrs(cnt[3]);
        std::vector<uint32_t> lens(cnt[3]);
        CDDT_CUDA(cudaMemcpyAsync(ptrs.data(), dptr.p, sizeof(unsigned long long) * cnt[3], cudaMemcpyDeviceToHost, st));
        CDDT_CUDA(cudaMemcpyAsync(lens.data(), dlen.p, sizeof(uint32_t) * cnt[3], cudaMemcpyDeviceToHost, st));
        CDDT_CUDA(cudaStreamSynchronize(st));
        uint32_t Pmax = 1;
        for (uint32_t n : lens) while (Pmax < n) Pmax <<= 1;
        Buf tmp;
        CDDT_CUDA(tmp.alloc(sizeof(KT) * (size_t)Pmax));
        for (uint32_t q = 0; q < cnt[3]; ++q) {
            uint32_t n = lens[q], P = 1;
            while (P < n) P <<= 1;
            KT *run = reinterpret_cast<KT *>((uintptr_t)ptrs[q]);
            copy_pad_kernel<KT><<<grid_for(P, 256), 256, 0, st>>>(run, n, tmp.as<KT>(), P);
            for (uint32_t k = 2; k <= P; k <<= 1)
                for (uint32_t j = k >> 1; j > 0; j >>= 1)
                    global_sort_stage_kernel<KT><<<grid_for(P, 256), 256, 0, st>>>(tmp.as<KT>(), P, k, j);
            copy_back_kernel<KT><<<grid_for(n, 256), 256, 0, st>>>(tmp.as<KT>(), n, run);
        }
    }
    CDDT_CUDA(cudaStreamSynchronize(st));
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

template cddt_status sort_segments<float>(const Segs<float> &, int64_t, cudaStream_t, Arena *);
template cddt_status sort_segments<uint16_t>(const Segs<uint16_t> &, int64_t, cudaStream_t, Arena *);

cddt_status index_store(cddt_s *h, cudaStream_t st)
{
    const int64_t nb = h->total_bins;
    if (h->u16) index_kernel<uint16_t><<<grid_for(nb * 32, 256), 256, 0, st>>>(h->store, h->hdr, nb);
    else index_kernel<float><<<grid_for(nb * 32, 256), 256, 0, st>>>(h->store, h->hdr, nb);
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}

// Sort every bin's leaf run (keys already scattered), pad and index.
cddt_status sort_and_index_any(cddt_s *h, cudaStream_t st)
{
    cddt_status rc;
    if (h->u16) {
        Segs<uint16_t> sg{h->store, h->hdr, nullptr, nullptr, nullptr};
        rc = sort_segments<uint16_t>(sg, h->total_bins, st);
    } else {
        Segs<float> sg{h->store, h->hdr, nullptr, nullptr, nullptr};
        rc = sort_segments<float>(sg, h->total_bins, st);
    }
    if (rc != CDDT_OK) return rc;
    return index_store(h, st);
}

// Lay out bins from per-bin counts: node offsets, bins[], store allocation.
// count_dev is consumed (overwritten).  Synchronises `st`.
cddt_status layout_bins(cddt_s *h, uint32_t *count_dev, cudaStream_t st, void **store_out,
                        int64_t *nodes_out, int64_t extra_nodes, Arena *ws, void **spare, int64_t *spare_nodes)
{
    int64_t nb = h->total_bins;
    const int LK = h->u16 ? 4 : 3;
    Buf nodes_b, scratch_b, zscratch_b, tot_b;
    uint32_t *nodes = nullptr;
    uint64_t *scratch = nullptr, *zscratch = nullptr, *tot = nullptr;
    if (ws) {
        nodes = ws->take<uint32_t>((size_t)nb);
        scratch = ws->take<uint64_t>((size_t)scan_scratch_elems(nb));
        zscratch = ws->take<uint64_t>((size_t)scan_scratch_elems(nb));
        tot = ws->take<uint64_t>(3);
    }
    if (!nodes || !scratch || !zscratch || !tot) {
        CDDT_CUDA(nodes_b.alloc(sizeof(uint32_t) * (size_t)nb));
        CDDT_CUDA(scratch_b.alloc(sizeof(uint64_t) * (size_t)scan_scratch_elems(nb)));
        CDDT_CUDA(zscratch_b.alloc(sizeof(uint64_t) * (size_t)scan_scratch_elems(nb)));
        CDDT_CUDA(tot_b.alloc(sizeof(uint64_t) * 3));
        nodes = nodes_b.as<uint32_t>();
        scratch = scratch_b.as<uint64_t>();
        zscratch = zscratch_b.as<uint64_t>();
        tot = tot_b.as<uint64_t>();
    }
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(tot + 2);
    CDDT_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    if (LK == 3) nodes_kernel<3, KeyT<float>::R><<<grid_for(nb, 256), 256, 0, st>>>(count_dev, nb, nodes);
    else nodes_kernel<4, KeyT<uint16_t>::R><<<grid_for(nb, 256), 256, 0, st>>>(count_dev, nb, nodes);
    exclusive_scan_u32(nodes, nodes, nb, scratch, tot, st);
    // total zero points: reduce the counts too
    {
        int64_t nblk = (nb + kScanTile - 1) / kScanTile;
        if (nblk) {
            scan_reduce_kernel<<<(unsigned)nblk, kScanThreads, 0, st>>>(count_dev, nb, zscratch);
            scan_partials_kernel<<<1, 1024, 0, st>>>(zscratch, nblk, tot + 1);
        } else {
            CDDT_CUDA(cudaMemsetAsync(tot + 1, 0, sizeof(uint64_t), st));
        }
    }
    hdr_kernel<<<grid_for(nb, 256), 256, 0, st>>>(count_dev, nodes, nb, h->hdr, mx);
    uint64_t host_tot[3];
    CDDT_CUDA(cudaMemcpyAsync(host_tot, tot, sizeof(host_tot), cudaMemcpyDeviceToHost, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    CDDT_CUDA(cudaGetLastError());
    if (host_tot[0] + (uint64_t)extra_nodes > 0xffffffffull) return CDDT_ERR_OOM;
    if (host_tot[2] > kMaxBinKeys) return CDDT_ERR_ARG;
    const int64_t need = std::max<int64_t>((int64_t)host_tot[0], 1);
    void *store = nullptr;
    if (spare && *spare && *spare_nodes >= need) {
        store = *spare;
        *spare = nullptr;
    } else {
        if (spare && *spare) {
            cudaFree(*spare);
            *spare = nullptr;
        }
        const int64_t alloc_nodes = need + extra_nodes;
        CDDT_CUDA(cudaMalloc(&store, (size_t)alloc_nodes * 32));
        if (spare_nodes) *spare_nodes = alloc_nodes;
    }
    *store_out = store;
    *nodes_out = (int64_t)host_tot[0];
    h->n_zp = (int64_t)host_tot[1];
    h->max_bin = (int64_t)host_tot[2];
    return CDDT_OK;
}

// Slice tables (readings S1-S3, S7), computed in double on the host.
static void slice_tables(cddt_s *h, std::vector<SliceInfo> &out)
{
    const double PI = 3.14159265358979323846;
    out.resize(h->S);
    double cx[4] = {-0.5, h->W - 0.5, -0.5, h->W - 0.5};
    double cy[4] = {-0.5, -0.5, h->H - 0.5, h->H - 0.5};
    uint32_t base = 0;
    for (int s = 0; s < h->S; ++s) {
        double ang = (2.0 * PI * (double)s) / (double)h->N;
        float c = (float)std::cos(ang), sn = (float)std::sin(ang);
        if (s == 0) { c = 1.0f; sn = 0.0f; }
        if (4 * s == h->N) { c = 0.0f; sn = 1.0f; }
        double ymin = 1e300, ymax = -1e300, xmin = 1e300;
        for (int q = 0; q < 4; ++q) {
            double yr = cy[q] * (double)c - cx[q] * (double)sn;
            double xr = cx[q] * (double)c + cy[q] * (double)sn;
            ymin = std::min(ymin, yr);
            ymax = std::max(ymax, yr);
            xmin = std::min(xmin, xr);
        }
        SliceInfo si{};
        si.c = c;
        si.s = sn;
        double T = std::ceil(-ymin) + 1.0;
        si.T = (int32_t)T;
        si.nb = (int32_t)(std::ceil(ymax + T) + 2.0);
        si.sbase = base;
        si.Tnb = (uint32_t)si.T | ((uint32_t)si.nb << 16);
        si.X = (float)(std::ceil(-xmin) + 1.0);
        base += (uint32_t)si.nb;
        out[s] = si;
    }
    h->total_bins = base;
}

// Build the store from the handle's edge map (used by build and by the
// update's rebuild-free path for tests).
cddt_status construct(cddt_s *h, cudaStream_t st)
{
    const int64_t ncell = (int64_t)h->W * h->H;
    const int threads = 256;
    // edge cell list
    int64_t nblk = (ncell + threads - 1) / threads;
    Buf bcount, boff, scratch, tot, cells;
    CDDT_CUDA(bcount.alloc(sizeof(uint32_t) * (size_t)nblk));
    CDDT_CUDA(boff.alloc(sizeof(uint32_t) * (size_t)nblk));
    CDDT_CUDA(scratch.alloc(sizeof(uint64_t) * (size_t)scan_scratch_elems(nblk)));
    CDDT_CUDA(tot.alloc(sizeof(uint64_t)));
    flag_count_kernel<<<(unsigned)nblk, threads, 0, st>>>(h->edge, ncell, bcount.as<uint32_t>());
    exclusive_scan_u32(bcount.as<uint32_t>(), boff.as<uint32_t>(), nblk, scratch.as<uint64_t>(), tot.as<uint64_t>(), st);
    uint64_t E = 0;
    CDDT_CUDA(cudaMemcpyAsync(&E, tot.p, sizeof(E), cudaMemcpyDeviceToHost, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    h->n_edge = (int64_t)E;
    CDDT_CUDA(cells.alloc(sizeof(uint32_t) * (size_t)std::max<uint64_t>(E, 1)));
    flag_write_kernel<<<(unsigned)nblk, threads, 0, st>>>(h->edge, ncell, boff.as<uint32_t>(), cells.as<uint32_t>());
    // counts
    Buf count;
    CDDT_CUDA(count.alloc(sizeof(uint32_t) * (size_t)h->total_bins));
    CDDT_CUDA(cudaMemsetAsync(count.p, 0, sizeof(uint32_t) * (size_t)h->total_bins, st));
    int64_t work = (int64_t)E * h->S;
    if (work) count_kernel<<<grid_for(work, threads), threads, 0, st>>>(cells.as<uint32_t>(), (int64_t)E, h->W, h->slices, h->S, count.as<uint32_t>());
    void *store = nullptr;
    int64_t nodes = 0;
    cddt_status rc = layout_bins(h, count.as<uint32_t>(), st, &store, &nodes, 0);
    if (rc != CDDT_OK) return rc;
    if (h->store) cudaFree(h->store);
    h->store = store;
    h->store_nodes = nodes;
    h->store_cap = std::max<int64_t>(nodes, 1);
    // scatter
    CDDT_CUDA(cudaMemsetAsync(count.p, 0, sizeof(uint32_t) * (size_t)h->total_bins, st));
    if (work) {
        if (h->u16)
            scatter_kernel<uint16_t><<<grid_for(work, threads), threads, 0, st>>>(cells.as<uint32_t>(), (int64_t)E, h->W, h->slices, h->S, h->hdr, count.as<uint32_t>(), h->store, h->Q);
        else
            scatter_kernel<float><<<grid_for(work, threads), threads, 0, st>>>(cells.as<uint32_t>(), (int64_t)E, h->W, h->slices, h->S, h->hdr, count.as<uint32_t>(), h->store, h->Q);
    }
    CDDT_CUDA(cudaGetLastError());
    rc = sort_and_index_any(h, st);
    if (rc != CDDT_OK) return rc;
    CDDT_CUDA(cudaStreamSynchronize(st));
    return CDDT_OK;
}

cddt_status init_handle(cddt_s *h, const uint8_t *grid_dev, cudaStream_t st, bool build)
{
    std::vector<SliceInfo> tab;
    slice_tables(h, tab);
    if (h->total_bins > 0xffffffffll) return CDDT_ERR_ARG;
    if (h->u16) {
        double diag = std::sqrt((double)h->W * h->W + (double)h->H * h->H);
        double q = 65535.0 / (diag + 4.0);
        if (q < 1.0) return CDDT_ERR_ARG;
        int e;
        std::frexp(q, &e);
        h->Q = (float)std::ldexp(1.0, e - 1);
        h->invQ = (float)(1.0 / std::ldexp(1.0, e - 1));
    }
    const int64_t ncell = (int64_t)h->W * h->H;
    CDDT_CUDA(cudaMalloc(&h->slices, sizeof(SliceInfo) * h->S));
    CDDT_CUDA(cudaMalloc(&h->hdr, sizeof(BinHdr) * (size_t)std::max<int64_t>(h->total_bins, 1)));
    CDDT_CUDA(cudaMalloc(&h->grid, (size_t)ncell));
    CDDT_CUDA(cudaMalloc(&h->edge, (size_t)ncell));
    CDDT_CUDA(cudaMalloc(&h->status, sizeof(int)));
    CDDT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CDDT_CUDA(cudaMemcpyAsync(h->slices, tab.data(), sizeof(SliceInfo) * h->S, cudaMemcpyHostToDevice, st));
    normalise_grid_kernel<<<grid_for(ncell, 256), 256, 0, st>>>(grid_dev, h->grid, ncell);
    edge_map_kernel<<<grid_for(ncell, 256), 256, 0, st>>>(h->grid, h->edge, h->W, h->H);
    CDDT_CUDA(cudaGetLastError());
    return build ? construct(h, st) : CDDT_OK;
}

// One warp per bin: its keys from an exported CSR into its leaf run (16-bit
// keys re-quantised, which restores them exactly); a bin that is not sorted
// ascending flags CDDT_ERR_DEVICE.
template <typename KT>
__global__ void load_bins_kernel(const float *zp, const uint32_t *start, const float *bin_X, const BinHdr *hdr,
                                 void *store, int64_t nbins, float Q, int *status)
{
    const int lane = threadIdx.x & 31;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t n = bin_count(hdr[g].nm);
        if (n == 0) continue;
        KT *run = leaf_run<KT>(store, hdr[g].off, n);
        const float *src = zp + start[g];
        for (uint32_t i = lane; i < n; i += 32) {
            const float v = src[i];
            if (i > 0 && !(src[i - 1] <= v)) atomicCAS(status, 0, (int)CDDT_ERR_DEVICE);
            if (sizeof(KT) == 4) reinterpret_cast<float *>(run)[i] = v;
            else reinterpret_cast<uint16_t *>(run)[i] = quantise(v, bin_X[g], Q);
        }
    }
}

cddt_status import_store(cddt_s *h, const int64_t *bin_start_host, const float *zp_host, cudaStream_t st)
{
    const int64_t nb = h->total_bins;
    if (bin_start_host[0] != 0) return CDDT_ERR_ARG;
    std::vector<uint32_t> cnt((size_t)std::max<int64_t>(nb, 1)), start((size_t)std::max<int64_t>(nb, 1));
    for (int64_t g = 0; g < nb; ++g) {
        const int64_t a = bin_start_host[g], b = bin_start_host[g + 1];
        if (b < a || b - a > (int64_t)kMaxBinKeys || b > 0xffffffffll) return CDDT_ERR_ARG;
        cnt[g] = (uint32_t)(b - a);
        start[g] = (uint32_t)a;
    }
    const int64_t n = bin_start_host[nb];
    std::vector<float> bin_X;
    if (h->u16) {
        std::vector<SliceInfo> tab;
        slice_tables(h, tab);
        bin_X.resize((size_t)std::max<int64_t>(nb, 1));
        for (int s = 0; s < h->S; ++s)
            for (int b = 0; b < tab[s].nb; ++b) bin_X[tab[s].sbase + b] = tab[s].X;
    }
    Buf cnt_d, start_d, zp_d, x_d;
    CDDT_CUDA(cnt_d.alloc(sizeof(uint32_t) * cnt.size()));
    CDDT_CUDA(start_d.alloc(sizeof(uint32_t) * start.size()));
    CDDT_CUDA(zp_d.alloc(sizeof(float) * (size_t)std::max<int64_t>(n, 1)));
    CDDT_CUDA(cudaMemcpyAsync(cnt_d.p, cnt.data(), sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st));
    CDDT_CUDA(cudaMemcpyAsync(start_d.p, start.data(), sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st));
    if (n) CDDT_CUDA(cudaMemcpyAsync(zp_d.p, zp_host, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    if (h->u16) {
        CDDT_CUDA(x_d.alloc(sizeof(float) * bin_X.size()));
        CDDT_CUDA(cudaMemcpyAsync(x_d.p, bin_X.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, st));
    }
    void *store = nullptr;
    int64_t nodes = 0;
    CDDT_TRY(layout_bins(h, cnt_d.as<uint32_t>(), st, &store, &nodes, 0));
    h->store = store;
    h->store_nodes = nodes;
    h->store_cap = std::max<int64_t>(nodes, 1);
    const unsigned blocks = grid_for(nb * 32, 256);
    if (h->u16)
        load_bins_kernel<uint16_t><<<blocks, 256, 0, st>>>(zp_d.as<float>(), start_d.as<uint32_t>(), x_d.as<float>(),
                                                            h->hdr, h->store, nb, h->Q, h->status);
    else
        load_bins_kernel<float><<<blocks, 256, 0, st>>>(zp_d.as<float>(), start_d.as<uint32_t>(), nullptr, h->hdr,
                                                         h->store, nb, h->Q, h->status);
    CDDT_CUDA(cudaGetLastError());
    CDDT_TRY(index_store(h, st));
    CDDT_CUDA(cudaStreamSynchronize(st));  // the host staging buffers are freed on return
    return CDDT_OK;
}

}  // namespace cddt
