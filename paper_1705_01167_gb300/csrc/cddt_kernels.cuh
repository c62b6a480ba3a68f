// cddt_kernels.cuh -- host-side entry points shared between the translation
// units of libcddt.so (scan, layout, sort/index, construction).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cddt_internal.cuh"

namespace cddt {

struct Arena;

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *scratch,
                        uint64_t *total_dev, cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);
// Lay out bins of the given key counts: headers (off, count) into h->hdr,
// and a store of at least that many nodes.  Temporaries come from `ws` when
// given.  Without `spare` a new store of nodes + extra_nodes is allocated.
// With `spare`, *spare (a buffer of *spare_nodes nodes, or null) is used
// when large enough (*spare becomes null), else it is freed and a new
// store with extra_nodes headroom allocated; *spare_nodes then receives the
// capacity of the returned store.
cddt_status layout_bins(cddt_s *h, uint32_t *count_dev, cudaStream_t st, void **store_out,
                        int64_t *nodes_out, int64_t extra_nodes, Arena *ws = nullptr, void **spare = nullptr,
                        int64_t *spare_nodes = nullptr);
cddt_status sort_and_index_any(cddt_s *h, cudaStream_t st);
cddt_status construct(cddt_s *h, cudaStream_t st);
// Slice tables, grid and edge map of a new handle, then (build) the store.
cddt_status init_handle(cddt_s *h, const uint8_t *grid_dev, cudaStream_t st, bool build = true);
// The store of an initialised handle from an exported CSR (cddt_import).
cddt_status import_store(cddt_s *h, const int64_t *bin_start_host, const float *zp_host, cudaStream_t st);
cddt_status prune(cddt_s *h, cudaStream_t st);
cddt_status update_cells(cddt_s *h, const int32_t *xy, const uint8_t *occ, int32_t n,
                         cudaStream_t st);

// Arguments of the sensor-model kernels (cddt_query.cu).
struct SensorArgs {
    const float *part;
    int64_t P;
    const float *beam_off;
    const float *obs;
    int32_t B, D;
    BeamConsts bc;
    float *logw;
    float *ranges;
    const float *grad_logw;
    float *grad_xy;
    unsigned long long *work;  // work-count mode: 6 counters
    float *part_out;           // refined poses (plan refinement)
};
cddt_status launch_sensor(const cddt_s *h, const SensorArgs &a, int mode, cudaStream_t st);
cddt_status calc_range(cddt_s *h, const float *pose, float *out, int64_t n, int sorted, cudaStream_t st);
cddt_status calc_range_timed(cddt_s *h, const float *pose, float *out, int64_t n, long long *cycles,
                             cudaStream_t st);
// The slice sort of cddt_calc_range_many (cddt_query.cu): blocks of
// kSortThreads threads place tiles of kSortTile queries; slices are grouped
// into at most kMaxSortBuckets buckets.
constexpr int kSortThreads = 512;
constexpr int kSortPerThread = 4;
constexpr int kSortTile = kSortThreads * kSortPerThread;
constexpr int kMaxSortBuckets = 1024;
// The slice-sorted cast on caller-provided scratch of sorted_scratch_bytes(h, n)
// bytes (cddt_query.cu); returns CDDT_ERR_ARG when the scratch is too small.
int64_t sorted_scratch_bytes(const cddt_s *h, int64_t n);
cddt_status calc_range_sorted_into(cddt_s *h, const float *pose, float *out, int64_t n, void *scratch,
                                   int64_t scratch_bytes, cudaStream_t st);

// Bump allocation from a caller-owned device buffer (256-byte aligned
// pieces); take() returns nullptr when the buffer is too small.
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    template <typename T> T *take(size_t n)
    {
        const size_t b = (n * sizeof(T) + 255) & ~(size_t)255;
        if (used + b > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += b;
        return p;
    }
    static size_t need(size_t bytes) { return (bytes + 255) & ~(size_t)255; }
};

// A device buffer freed on scope exit.
struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
    template <typename T> T *as() { return reinterpret_cast<T *>(p); }
};

template <typename KT> __device__ __forceinline__ KT pad_key();
template <> __device__ __forceinline__ float pad_key<float>() { return kInf; }
template <> __device__ __forceinline__ uint16_t pad_key<uint16_t>() { return 0xffffu; }

// First key of a bin's leaf run.
template <typename KT>
__device__ __forceinline__ KT *leaf_run(void *store, uint32_t off, uint32_t n)
{
    constexpr int LK = KeyT<KT>::LK;
    return reinterpret_cast<KT *>(store) + ((size_t)(off + internal_nodes(n, LK, KeyT<KT>::R)) << LK);
}

// The segments of a segmented sort: the leaf runs of a store's bins (hdr
// set), or plain ranges base[off[id] .. off[id] + len[id]).
template <typename KT>
struct Segs {
    void *store;
    const BinHdr *hdr;
    KT *base;
    const uint32_t *off;
    const uint32_t *len;
    // when skip_upto > 0, sort_segments leaves alone every segment of at most
    // skip_upto keys whose companion length (also_len, when given) is at
    // most skip_upto too
    const uint32_t *also_len = nullptr;
    uint32_t skip_upto = 0;
    __device__ __forceinline__ void get(uint32_t id, KT *&p, uint32_t &n) const
    {
        if (hdr) {
            n = bin_count(hdr[id].nm);
            p = leaf_run<KT>(store, hdr[id].off, n);
        } else {
            n = len[id];
            p = base + off[id];
        }
    }
};

// Sort every segment ascending (cddt_build.cu).  Synchronises `st`.
template <typename KT>
cddt_status sort_segments(const Segs<KT> &sg, int64_t nseg, cudaStream_t st, Arena *ws = nullptr);
// Fill the trees and headers of every bin from the sorted leaf runs.
cddt_status index_store(cddt_s *h, cudaStream_t st);
// Slice tables' eps for pruning: 32 units in the last place of the largest
// projected coordinate.
float prune_eps(int W, int H);

// Threads of a block of the gradient refinement kernels (cddt_plan_refine
// launches them with this size; the wider kernels size their shared sums by
// it).
constexpr int kRefineBlock = 256;

// Blocks of a grid-stride launch over n items: one per `threads` items, at
// most per_sm blocks per streaming multiprocessor.
inline unsigned grid_cap(int64_t n, int threads, int64_t per_sm = 64)
{
    const int64_t cap = (int64_t)sm_count() * per_sm;
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename KT>
__device__ __forceinline__ uint32_t key_bits(KT v)
{
    if (sizeof(KT) == 4) return __float_as_uint(*reinterpret_cast<const float *>(&v));
    return (uint32_t)(*reinterpret_cast<const uint16_t *>(&v));
}

// Index one bin whose sorted keys sit in its leaf run (W >= 8 lanes of a
// warp, lane = 0..W-1 among them, mask = their bits; by default the whole
// warp): pad the last leaf, fill the internal levels with the largest key
// under each child, and write the root separators (or the keys of a small
// bin) and the tree shape into the header.  The lanes' writes of the leaf
// run must be visible to all of them (a __syncwarp(mask) after writing them
// is enough).
template <typename KT, int W = 32>
__device__ __forceinline__ void index_bin(void *store, BinHdr *hdr, int64_t g, int lane,
                                          unsigned mask = 0xffffffffu)
{
    static_assert(W >= 8 && W <= 32, "index_bin needs 8 to 32 lanes");
    constexpr int LK = KeyT<KT>::LK;
    constexpr int R = KeyT<KT>::R;
    {
        const uint32_t n = bin_count(hdr[g].nm), off = hdr[g].off;
        if (n == 0) return;
        KT *run = reinterpret_cast<KT *>(store) + ((size_t)off << LK);
        const uint32_t L0 = ((n - 1) >> LK) + 1;
        const int h = run_levels(L0, LK, R);
        const uint32_t internal = internal_nodes(n, LK, R);
        KT *leaves = run + ((size_t)internal << LK);
        for (uint32_t i = n + lane; i < (L0 << LK); i += W) leaves[i] = pad_key<KT>();
        uint32_t loff = 0;
        for (int l = h; l >= 1; --l) {
            const uint32_t cnt = level_count(L0, LK, l);
            for (uint32_t slot = lane; slot < (cnt << LK); slot += W) {
                const uint64_t first = (uint64_t)slot << (LK * l);
                KT v = pad_key<KT>();
                if (first < n) {
                    uint64_t last = ((uint64_t)slot + 1) << (LK * l);
                    if (last > n) last = n;
                    v = leaves[last - 1];
                }
                run[((size_t)loff << LK) + slot] = v;
            }
            loff += cnt;
        }
        // header separators: R keys packed into 6 words
        if (lane < 6) {
            uint32_t word = 0;
            const uint32_t cnt_h = level_count(L0, LK, h);
            const int per = 4 / (int)sizeof(KT);  // keys per word
            for (int e = 0; e < per; ++e) {
                const uint32_t q = (uint32_t)(lane * per + e);
                KT v = pad_key<KT>();
                if (n <= (uint32_t)R) {
                    if (q < n) v = leaves[q];
                } else if (q < cnt_h) {
                    uint64_t last = ((uint64_t)q + 1) << (LK * (h + 1));
                    if (last > n) last = n;
                    v = leaves[last - 1];
                }
                word |= key_bits<KT>(v) << (16 * e);
            }
            hdr[g].w[lane] = word;
        }
        __syncwarp(mask);
        if (lane == 0) hdr[g].nm = n | ((uint32_t)h << 24) | (level_count(L0, LK, h) << 28);
    }
}


}  // namespace cddt
