// cddt_maintain.cu -- pruning (Section IV-C, PCDDT) and incremental cell
// updates (Section IV-D) of a built CDDT, on the GPU.
//
// Pruning keeps zero point z_m of a bin iff the closed gap [z_{m-1}, z_m]
// (used by forward queries) or [z_m, z_{m+1}] (used by backward queries)
// meets the x'-extent of a free in-map cell whose y'-extent meets the bin,
// both widened by eps; so no query from a free cell changes its answer.  In
// slice 0 the rotation is exact and a query's bin is exactly its row, so a
// row reaches only its own bin there.
//
// An update applies the cell writes (the last write to a cell wins),
// re-evaluates the edge status of every written cell and its 8 neighbours,
// turns each flip into +/- zero points in every overlapped bin of every
// slice, sorts the deltas of each bin and merges them into a new store (the
// old store is read once and the new one written once), then refills the
// search trees.  The result equals a build on the updated grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

float prune_eps(int W, int H)
{
    const double diag = std::sqrt((double)W * W + (double)H * H);
    const int e = (int)std::ceil(std::log2(2.0 * diag + 8.0));
    return (float)std::ldexp(1.0, e - 18);
}

// ------------------------------------------------------------ prune

// A stored key as the raw word the node comparisons take.
template <typename KT>
__device__ __forceinline__ uint32_t raw_key(const KT *leaves, int i)
{
    if (sizeof(KT) == 4) return __float_as_uint(__ldg(reinterpret_cast<const float *>(leaves) + i));
    return (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(leaves) + i);
}

// Marks of one free cell in one bin its extent reaches (reading S8): every
// key m in [lower_bound(xlo) - 1, upper_bound(xhi)], clamped to the bin,
// whose forward or backward gap meets the cell's widened x' extent.  The
// bin's leaf run (leaves, bn keys) and its marks (kp) come from the caller;
// lc holds a lower bound near the cell's (the search of its line), which
// moves by a key or two to the cell's own: the cells of a line lie within
// a unit of one another in x'.
template <typename KT>
__device__ __forceinline__ void prune_mark_cell(const MapView &m, uint32_t g, float X, float xlo, float xhi,
                                                uint64_t pol, const KT *leaves, int bn, uint8_t *kp, int &lc)
{
    const Cmp<KT, false> below(m, xlo, X);  // key < xlo, as in the tree search
    int l = lc;
    while (l > 0 && !below.le(raw_key<KT>(chk_store(m, leaves + l - 1, (int)sizeof(KT)), 0))) --l;
    while (l < bn && below.le(raw_key<KT>(chk_store(m, leaves + l, (int)sizeof(KT)), 0))) ++l;
    lc = l;  // first key >= xlo
    // first key > xhi: the cell's x' extent is under two units wide, so it
    // is usually within a few keys of l
    const Cmp<KT, true> above(m, xhi, X);
    int u = l;
    if (u < bn && above.le(raw_key<KT>(chk_store(m, leaves + u, (int)sizeof(KT)), 0))) {
        ++u;
        while (u < bn && u < l + 8 && above.le(raw_key<KT>(chk_store(m, leaves + u, (int)sizeof(KT)), 0))) ++u;
        if (u == l + 8) {
            int kb;
            u = bin_search<KT, true, CDDT_SEARCH_TREE>(m, g, xhi, X, pol, kb).idx;
        }
    }
    const int m1 = min(u, bn - 1);
    for (int mm = max(l - 1, 0); mm <= m1; ++mm) kp[mm] = 1;
}

// Prune marks, bin by bin: one warp per bin (s, b).  The free cells whose
// widened y' extent meets the bin lie in a strip along direction s; the
// lanes take consecutive lines of the strip (columns when |cos| >= sin,
// else rows), so that the warp's searches all run in one bin, whose header
// and nodes stay in L1.  Each line holds a few candidate cells: those whose
// y' lies in the bin's band widened by a margin (0.25) far above the float
// rounding of the candidate arithmetic; every candidate then takes the
// exact per-cell test of reading S8 (the bins b0..b1 of the cell, computed
// with the same float operations as the oracle), so each (free cell, bin)
// pair is marked exactly when the cell-by-cell rule marks it.  A line
// takes one tree search (at its first candidate's x') and its cells move
// from there.
template <typename KT>
__global__ void prune_mark_kernel(MapView m, float eps, uint8_t *keep, int64_t keep_n, int64_t total_bins)
{
    constexpr int LK = KeyT<KT>::LK;
    const uint64_t pol = policy_evict_last();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total_bins; g += nwarps) {
        int lo = 0, hi = m.S - 1;  // slice of bin g: the last s with sbase <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)__ldg(&m.slices[mid].sbase) <= g) lo = mid;
            else hi = mid - 1;
        }
        const int s = lo;
        const SliceInfo si = *chk_slice(m, m.slices + s, (int)sizeof(SliceInfo));
        const BinHdr bh = *chk_hdr(m, m.hdr + g, (int)sizeof(BinHdr));
        const int bn = (int)bin_count(bh.nm);
        if (bn == 0) continue;
        const int64_t k0 = ((int64_t)bh.off + internal_nodes((uint32_t)bn, LK, KeyT<KT>::R)) << LK;
#if CDDT_CHECKED
        if (k0 < 0 || k0 + bn > keep_n) {
            atomicCAS(m.status, 0, (int)CDDT_ERR_BOUNDS);
            continue;
        }
#else
        (void)keep_n;
#endif
        const KT *leaves = reinterpret_cast<const KT *>(m.store) + k0;
        uint8_t *kp = keep + k0;
        const int b = (int)(g - si.sbase);
        const float c = si.c, sn = si.s;
        const float h = half_extent(c, sn);
        // candidate band of y' = j c - i sn
        const float bp = (float)(b - si.T);
        const float ylo = bp - 0.5f - h - eps - 0.25f, yhi = bp + 0.5f + h + eps + 0.25f;
        const bool cols = fabsf(c) >= sn;
        const int L = cols ? m.W : m.H;
        // lines whose candidate range meets the map (one line of margin)
        float k_lo = 0.0f, k_hi = (float)(L - 1);
        if (cols) {  // j in [(ylo + i sn) / c, (yhi + i sn) / c] (ends swapped for c < 0)
            if (sn > 0.0f) {
                const float hc = (float)(m.H - 1) * c;
                if (c > 0.0f) { k_lo = -yhi / sn; k_hi = (hc - ylo) / sn; }
                else { k_lo = (hc - yhi) / sn; k_hi = -ylo / sn; }
            } else if (yhi < 0.0f || ylo > (float)(m.H - 1)) {
                continue;  // slice 0: the band misses every row
            }
        } else {  // i in [(j c - yhi) / sn, (j c - ylo) / sn]
            const float ws = (float)(m.W - 1) * sn;
            if (c > 0.0f) { k_lo = ylo / c; k_hi = (ws + yhi) / c; }
            else if (c < 0.0f) { k_lo = (ws + yhi) / c; k_hi = ylo / c; }
            else if (ylo > 0.0f || ws + yhi < 0.0f) continue;
        }
        const int l0 = max(0, (int)floorf(fmaxf(k_lo, -1.0f)) - 1);
        const int l1 = min(L - 1, (int)ceilf(fminf(k_hi, (float)L)) + 1);
        const float inv = 1.0f / (cols ? c : sn);
        for (int k = l0 + lane; k <= l1; k += 32) {
            int a0, a1;  // cells of line k: rows (cols) or columns
            if (cols) {
                const float p = ((float)k * sn + ylo) * inv, q = ((float)k * sn + yhi) * inv;
                a0 = max(0, (int)ceilf(fminf(p, q)));
                a1 = min(m.H - 1, (int)floorf(fmaxf(p, q)));
            } else {
                const float p = ((float)k * c - yhi) * inv, q = ((float)k * c - ylo) * inv;
                a0 = max(0, (int)ceilf(p));
                a1 = min(m.W - 1, (int)floorf(q));
            }
            int lc = 0;
            if (a0 <= a1) {  // the line's search, at its first candidate
                float xr, yr;
                project((float)(cols ? k : a0), (float)(cols ? a0 : k), c, sn, xr, yr);
                int kb;
                lc = bin_search<KT, false, CDDT_SEARCH_TREE>(m, (uint32_t)g, __fsub_rn(__fsub_rn(xr, h), eps), si.X,
                                                             pol, kb).idx;
            }
            for (int a = a0; a <= a1; ++a) {
                const int i = cols ? k : a, j = cols ? a : k;
                if (__ldg(m.grid + (int64_t)j * m.W + i)) continue;
                float xr, yr;
                project((float)i, (float)j, c, sn, xr, yr);
                int b0, b1;
                if (s == 0) {
                    b0 = b1 = j + si.T;
                } else {
                    const float clo = __fsub_rn(__fsub_rn(yr, h), eps), chi = __fadd_rn(__fadd_rn(yr, h), eps);
                    b0 = (int)ceilf(__fsub_rn(clo, 0.5f)) + si.T;
                    b1 = (int)floorf(__fadd_rn(chi, 0.5f)) + si.T;
                }
                b0 = max(b0, 0);
                b1 = min(b1, si.nb - 1);
                if (b < b0 || b > b1) continue;
                const float xlo = __fsub_rn(__fsub_rn(xr, h), eps), xhi = __fadd_rn(__fadd_rn(xr, h), eps);
                prune_mark_cell<KT>(m, (uint32_t)g, si.X, xlo, xhi, pol, leaves, bn, kp, lc);
            }
        }
    }
}

template <typename KT>
__global__ void count_kept_kernel(const BinHdr *hdr, int64_t nbins, const uint8_t *keep, uint32_t *cnt)
{
    constexpr int LK = KeyT<KT>::LK;
    const int lane = threadIdx.x & 31;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const BinHdr bh = hdr[g];
        const uint32_t bn = bin_count(bh.nm);
        const uint8_t *kp = keep + (((size_t)bh.off + internal_nodes(bn, LK, KeyT<KT>::R)) << LK);
        uint32_t c = 0;
        for (uint32_t i = lane; i < bn; i += 32) c += kp[i];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[g] = c;
    }
}

// Copy each bin's kept keys, in order, into the new store.
template <typename KT>
__global__ void compact_kernel(void *old_store, const BinHdr *old_hdr, const uint8_t *keep, void *new_store,
                               const BinHdr *new_hdr, int64_t nbins)
{
    constexpr int LK = KeyT<KT>::LK;
    const int lane = threadIdx.x & 31;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const BinHdr ob = old_hdr[g], nb = new_hdr[g];
        const uint32_t on = bin_count(ob.nm), nn = bin_count(nb.nm);
        const KT *src = leaf_run<KT>(old_store, ob.off, on);
        const uint8_t *kp = keep + (((size_t)ob.off + internal_nodes(on, LK, KeyT<KT>::R)) << LK);
        KT *dst = leaf_run<KT>(new_store, nb.off, nn);
        uint32_t o = 0;
        for (uint32_t i0 = 0; i0 < on; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool k = i < on && kp[i];
            const unsigned msk = __ballot_sync(0xffffffffu, k);
            if (k) {
                const uint32_t pos = o + __popc(msk & ((1u << lane) - 1));
                if (pos < nn) dst[pos] = src[i];
            }
            o += __popc(msk);
        }
    }
}

template <typename KT>
static cddt_status prune_kt(cddt_s *h, cudaStream_t st)
{
    constexpr int K = KeyT<KT>::K;
    const int64_t nb = h->total_bins;
    Buf keep, cnt, old_hdr;
    CDDT_CUDA(keep.alloc((size_t)h->store_nodes * K));
    CDDT_CUDA(cnt.alloc(sizeof(uint32_t) * (size_t)std::max<int64_t>(nb, 1)));
    CDDT_CUDA(old_hdr.alloc(sizeof(BinHdr) * (size_t)std::max<int64_t>(nb, 1)));
    CDDT_CUDA(cudaMemsetAsync(keep.p, 0, (size_t)h->store_nodes * K, st));
    prune_mark_kernel<KT><<<grid_cap(nb * 32, 256, 32), 256, 0, st>>>(h->view(), prune_eps(h->W, h->H),
                                                                        keep.as<uint8_t>(), h->store_nodes * K, nb);
    count_kept_kernel<KT><<<grid_cap(nb * 32, 256), 256, 0, st>>>(h->hdr, nb, keep.as<uint8_t>(), cnt.as<uint32_t>());
    CDDT_CUDA(cudaMemcpyAsync(old_hdr.p, h->hdr, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st));
    CDDT_CUDA(cudaGetLastError());
    void *store = nullptr;
    int64_t nodes = 0;
    cddt_status rc = layout_bins(h, cnt.as<uint32_t>(), st, &store, &nodes, 0);
    if (rc != CDDT_OK) {
        // the old headers are still valid for the old store
        cudaMemcpyAsync(h->hdr, old_hdr.p, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
        return rc;
    }
    compact_kernel<KT><<<grid_cap(nb * 32, 256), 256, 0, st>>>(h->store, old_hdr.as<BinHdr>(), keep.as<uint8_t>(), store,
                                                               h->hdr, nb);
    CDDT_CUDA(cudaGetLastError());
    CDDT_CUDA(cudaStreamSynchronize(st));
    cudaFree(h->store);
    h->store = store;
    h->store_nodes = nodes;
    h->store_cap = std::max<int64_t>(nodes, 1);
    rc = index_store(h, st);
    if (rc != CDDT_OK) return rc;
    CDDT_CUDA(cudaStreamSynchronize(st));
    return CDDT_OK;
}

cddt_status prune(cddt_s *h, cudaStream_t st)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    cddt_status rc = h->u16 ? prune_kt<uint16_t>(h, st) : prune_kt<float>(h, st);
    if (rc == CDDT_OK) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&h->prune_ms, e0, e1);
        h->pruned = 1;
    }
    h->generation++;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// ------------------------------------------------------------ update

__device__ __forceinline__ void flag_error(int *status) { atomicCAS(status, 0, (int)CDDT_ERR_DEVICE); }

__global__ void upd_dedupe_kernel(const int32_t *xy, int32_t n, int W, int H, int32_t *last, int *status)
{
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int x = xy[2 * t], y = xy[2 * t + 1];
        if (x < 0 || x >= W || y < 0 || y >= H) {
            flag_error(status);
            continue;
        }
        atomicMax(last + (int64_t)y * W + x, t);
    }
}

// The last write to each cell applies; the cell's marker returns to -1.
__global__ void upd_apply_kernel(const int32_t *xy, const uint8_t *occ, int32_t n, int W, int H, int32_t *last,
                                 uint8_t *grid, uint32_t *changed, uint32_t *nchanged)
{
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int x = xy[2 * t], y = xy[2 * t + 1];
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        const int64_t q = (int64_t)y * W + x;
        if (last[q] != t) continue;
        last[q] = -1;
        const uint8_t nv = occ[t] ? 1 : 0;
        if (grid[q] != nv) {
            grid[q] = nv;
            changed[atomicAdd(nchanged, 1u)] = (uint32_t)q;
        }
    }
}

// Edge-status flips in the 3x3 neighbourhood of every changed cell (each
// cell examined once per update through an epoch stamp).
__global__ void upd_flip_kernel(const uint32_t *changed, const uint32_t *nchanged, int W, int H, const uint8_t *grid,
                                uint8_t *edge, uint32_t *stamp, uint32_t epoch, uint32_t *flips, uint32_t *nflips)
{
    const uint32_t nc = *nchanged;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const uint32_t q = changed[c];
        const int j = (int)(q / (uint32_t)W), i = (int)(q - (uint32_t)j * W);
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int a = i + di, b = j + dj;
                if (a < 0 || a >= W || b < 0 || b >= H) continue;
                const uint32_t qq = (uint32_t)b * W + a;
                if (atomicExch(stamp + qq, epoch) == epoch) continue;
                const uint8_t e = edge_at(grid, W, H, a, b);
                if (e != edge[qq]) {
                    edge[qq] = e;
                    flips[atomicAdd(nflips, 1u)] = qq | (e ? 0x80000000u : 0u);
                }
            }
    }
}

// Pass 0 counts the +/- zero points of every flip per bin; pass 1 scatters
// them into per-bin segments.
template <typename KT, int PASS>
__global__ void upd_delta_kernel(const uint32_t *flips, const uint32_t *nflips, int W, const SliceInfo *slices, int S,
                                 float Q, uint32_t *ins_n, uint32_t *del_n, const uint32_t *ins_off,
                                 const uint32_t *del_off, KT *ins_keys, KT *del_keys, uint32_t *ins_bin,
                                 uint32_t *del_bin)
{
    const int64_t total = (int64_t)(*nflips) * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t % S);
        const uint32_t v = flips[t / S];
        const bool ins = (v >> 31) != 0;
        const uint32_t q = v & 0x7fffffffu;
        const int j = (int)(q / (uint32_t)W), i = (int)(q - (uint32_t)j * W);
        const SliceInfo si = slices[s];
        float xr, yr;
        project((float)i, (float)j, si.c, si.s, xr, yr);
        int b0, b1;
        if (!cell_bins(yr, half_extent(si.c, si.s), si.T, si.nb, b0, b1)) continue;
        KT key;
        if (sizeof(KT) == 4) *reinterpret_cast<float *>(&key) = xr;
        else *reinterpret_cast<uint16_t *>(&key) = quantise(xr, si.X, Q);
        for (int b = b0; b <= b1; ++b) {
            const uint32_t g = si.sbase + (uint32_t)b;
            if (PASS == 0) {
                atomicAdd(ins ? ins_n + g : del_n + g, 1u);
            } else {
                // ins_n / del_n are cursors here (zeroed before this pass)
                if (ins) {
                    const uint32_t t = ins_off[g] + atomicAdd(ins_n + g, 1u);
                    ins_keys[t] = key;
                    ins_bin[t] = g;
                } else {
                    const uint32_t t = del_off[g] + atomicAdd(del_n + g, 1u);
                    del_keys[t] = key;
                    del_bin[t] = g;
                }
            }
        }
    }
}

__global__ void upd_newcount_kernel(const BinHdr *hdr, const uint32_t *ins_n, const uint32_t *del_n, int64_t nbins,
                                    uint32_t *new_n, int *status)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nbins;
         g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t n = bin_count(hdr[g].nm), d = del_n[g];
        if (d > n) flag_error(status);
        new_n[g] = n + ins_n[g] - min(d, n);
    }
}

template <typename KT>
__device__ __forceinline__ int lower_bound_k(const KT *a, int n, KT v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
template <typename KT>
__device__ __forceinline__ int upper_bound_k(const KT *a, int n, KT v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(v < a[mid])) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Number of a node's stored keys below v (raw key order), over words
// [from, 8): one key per word for float32, two for 16-bit keys.
template <typename KT>
__device__ __forceinline__ int raw_count_lt(const uint32_t (&w)[8], int from, KT v)
{
    int c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < from) continue;
        if (sizeof(KT) == 4) c += __uint_as_float(w[i]) < *reinterpret_cast<const float *>(&v);
        else {
            const uint32_t x = (uint32_t)*reinterpret_cast<const uint16_t *>(&v);
            c += (w[i] & 0xffffu) < x;
            c += (w[i] >> 16) < x;
        }
    }
    return c;
}

// lower_bound (the number of keys below v) in a bin of an indexed store,
// through its header and tree: one node per level instead of a binary
// search's log2(n) dependent probes.
template <typename KT>
__device__ __forceinline__ int tree_lower_bound(const void *store, const BinHdr &hb, KT v)
{
    constexpr int LK = KeyT<KT>::LK;
    constexpr int K = KeyT<KT>::K;
    constexpr int R = KeyT<KT>::R;
    const uint32_t n = bin_count(hb.nm);
    if (n == 0) return 0;
    uint32_t w[8] = {hb.off, hb.nm, hb.w[0], hb.w[1], hb.w[2], hb.w[3], hb.w[4], hb.w[5]};
    int c = raw_count_lt<KT>(w, 2, v);
    if (n <= (uint32_t)R) return min(c, (int)n);
    const uint32_t L0 = ((n - 1) >> LK) + 1;
    const int h = (int)((hb.nm >> 24) & 15u);
    const int cnt_h = (int)(hb.nm >> 28);
    if (c >= cnt_h) return (int)n;
    const char *run = reinterpret_cast<const char *>(store) + ((size_t)hb.off << 5);
    uint32_t loff = 0, k = (uint32_t)c, cnt = (uint32_t)cnt_h;
    for (int l = h; l >= 1; --l) {
        ld_node(run + ((size_t)(loff + k) << 5), w);
        const int cc = raw_count_lt<KT>(w, 0, v);
        loff += cnt;
        cnt = ((L0 - 1) >> (LK * (l - 1))) + 1;
        k = min(k * K + (uint32_t)cc, cnt - 1);
    }
    ld_node(run + ((size_t)(loff + k) << 5), w);
    return min((int)(k * K) + raw_count_lt<KT>(w, 0, v), (int)n);
}

__device__ __forceinline__ uint32_t key_word(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t key_word(uint16_t v) { return (uint32_t)v; }
__device__ __forceinline__ float shfl_key(float v, int k) { return __shfl_sync(0xffffffffu, v, k); }
__device__ __forceinline__ uint16_t shfl_key(uint16_t v, int k)
{
    return (uint16_t)__shfl_sync(0xffffffffu, (uint32_t)v, k);
}
// Ballot over a group of W lanes (mask = the group's lanes): bit k for the
// group's lane k.
template <int W>
__device__ __forceinline__ uint32_t group_ballot(unsigned mask, bool p)
{
    const uint32_t b = __ballot_sync(mask, p);
    if (W == 32) return b;
    return (b >> (threadIdx.x & 31 & ~(W - 1))) & ((1u << W) - 1u);
}
// The same within groups of W lanes (mask = the group's lanes).
template <int W>
__device__ __forceinline__ float shfl_key_w(unsigned mask, float v, int k) { return __shfl_sync(mask, v, k, W); }
template <int W>
__device__ __forceinline__ uint16_t shfl_key_w(unsigned mask, uint16_t v, int k)
{
    return (uint16_t)__shfl_sync(mask, (uint32_t)v, k, W);
}

// After the per-bin sort of the deltas: for every insert, the number of old
// keys below it (lower_bound in its bin); for every delete, the index of the
// old key it removes (lower_bound plus its rank among equal deletes of the
// bin).  One thread per delta, each a tree search of the old store.
template <typename KT>
__global__ void upd_locate_kernel(const KT *keys, const uint32_t *bins, const uint32_t *seg_off,
                                  const uint32_t *seg_len, const uint32_t *also_len, int64_t total, bool deletes,
                                  const void *old_store, const BinHdr *old_hdr, int32_t *pos, int *status)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = bins[t];
        const KT key = keys[t];
        const BinHdr ob = old_hdr[g];
        int p = tree_lower_bound<KT>(old_store, ob, key);
        if (deletes) {
            // rank among the bin's equal deletes (any order of them is fine:
            // equal deletes remove distinct equal keys)
            const int64_t first = seg_off[g];
            if (seg_len[g] > 32 || also_len[g] > 32)  // sorted: equal deletes are adjacent
                for (int64_t u = t - 1; u >= first && keys[u] == key; --u) ++p;
            else
                for (int64_t u = first; u < t; ++u) p += keys[u] == key;
            const uint32_t n = bin_count(ob.nm);
            if (p >= (int)n || leaf_run<KT>(const_cast<void *>(old_store), ob.off, n)[p] != key) {
                flag_error(status);  // a delete with no key to remove
                p = 0x7fffffff;
            }
        }
        pos[t] = p;
    }
}

// Merge each bin's old sorted keys with its sorted inserts, dropping one
// occurrence per delete.  For an old key v at index i (first occurrence a):
// it is deleted iff i - a < (#deletes equal to v); a kept key lands at
// i - #(deletes <= v) + #(inserts <= v).  An insert u at index j lands at
// j + #(old < u) - #(deletes < u).  (Inserts precede equal old keys.)
template <typename KT>
__device__ __forceinline__ void merge_bin(const void *old_store, const BinHdr *old_hdr, void *new_store,
                                          const BinHdr *new_hdr, const KT *ins_keys, const uint32_t *ins_off,
                                          const uint32_t *ins_n, const KT *del_keys, const uint32_t *del_off,
                                          const uint32_t *del_n, const int32_t *ins_lb, const int32_t *del_pos,
                                          int64_t g, int lane, int *status)
{
    {
        const BinHdr ob = old_hdr[g], nb = new_hdr[g];
        const uint32_t obn = bin_count(ob.nm), nbn = bin_count(nb.nm);
        const KT *old = leaf_run<KT>(const_cast<void *>(old_store), ob.off, obn);
        KT *dst = leaf_run<KT>(new_store, nb.off, nbn);
        const int n = (int)obn, ni = (int)ins_n[g], nd = (int)min(del_n[g], obn), nn = (int)nbn;
        const KT *I = ins_keys + ins_off[g];
        const KT *Dl = del_keys + del_off[g];
        // 16-byte pieces: leaf runs are 32-byte aligned and padded to whole
        // leaves, so a piece that starts below n lies inside the run
        constexpr int V = 16 / (int)sizeof(KT);
        if (ni == 0 && nd == 0) {
            if (n == nn)
                for (int i = lane * V; i < n; i += 32 * V)
                    *reinterpret_cast<uint4 *>(dst + i) = __ldg(reinterpret_cast<const uint4 *>(old + i));
            else
                flag_error(status);
            return;
        }
        if (ni <= 32 && nd <= 32) {
            // Few changes (the common case): lane k holds insert k (with the
            // number of old keys below it) and the old index that delete k
            // removes.  A kept old key at index i moves to i - #(deletes
            // placed before i) + #(inserts <= its value), and insert j to
            // j + #(old < u_j) - #(deletes < u_j) (inserts precede equal old
            // keys).
            const KT ik = lane < ni ? I[lane] : KT(0);
            const int ilb = lane < ni ? ins_lb[ins_off[g] + lane] : 0;
            const int dpos = lane < nd ? del_pos[del_off[g] + lane] : 0x7fffffff;
            // each lane takes U 16-byte pieces of V keys per pass (8 keys)
            constexpr int U = 8 / V > 0 ? 8 / V : 1;
            for (int i0 = 0; i0 < n; i0 += 32 * V * U) {
                KT v[U][V];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ib = i0 + (u * 32 + lane) * V;
                    uint4 q = make_uint4(0u, 0u, 0u, 0u);
                    if (ib < n) q = __ldg(reinterpret_cast<const uint4 *>(old + ib));
                    memcpy(v[u], &q, 16);
                }
                int dbefore[U][V], ibefore[U][V];
                bool gone[U][V];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        dbefore[u][e] = 0;
                        ibefore[u][e] = 0;
                        gone[u][e] = false;
                    }
                for (int k = 0; k < nd; ++k) {
                    const int pk = __shfl_sync(0xffffffffu, dpos, k);
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const int i = i0 + (u * 32 + lane) * V + e;
                            dbefore[u][e] += pk < i;
                            gone[u][e] |= pk == i;
                        }
                }
                for (int k = 0; k < ni; ++k) {
                    const KT uk = shfl_key(ik, k);
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int e = 0; e < V; ++e) ibefore[u][e] += !(v[u][e] < uk);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int i = i0 + (u * 32 + lane) * V + e;
                        if (i < n && !gone[u][e]) {
                            const int pos = i - dbefore[u][e] + ibefore[u][e];
                            if (pos < 0 || pos >= nn) flag_error(status);
                            else dst[pos] = v[u][e];
                        }
                    }
            }
            // inserts in any order: insert j's rank among the bin's inserts
            int jr = 0;
            for (int k = 0; k < ni; ++k) {
                const KT uk = shfl_key(ik, k);
                jr += (uk < ik) || (uk == ik && k < lane);
            }
            if (lane < ni) {
                int dlt = 0;  // deletes below the insert
                for (int k = 0; k < nd; ++k) dlt += Dl[k] < ik;
                const int pos = jr + ilb - dlt;
                if (pos < 0 || pos >= nn) flag_error(status);
                else dst[pos] = ik;
            }
            return;
        }
        // Many changes (inserts and deletes sorted, delete positions
        // ascending): the run is streamed in chunks like above, and each chunk
        // counts only the deletes placed inside it and the inserts between its
        // first and last key; everything before the chunk is a base count.
        const int32_t *DP = del_pos + del_off[g];
        const int32_t *IL = ins_lb + ins_off[g];
        constexpr int U = 8 / V > 0 ? 8 / V : 1;
        constexpr int C = 32 * V * U;  // keys per chunk
        for (int i0 = 0; i0 < n; i0 += C) {
            const int iend = min(i0 + C, n);
            const int d_lo = lower_bound_k<int32_t>(DP, nd, i0), d_hi = lower_bound_k<int32_t>(DP, nd, iend);
            const int i_lo = lower_bound_k<KT>(I, ni, old[i0]), i_hi = upper_bound_k<KT>(I, ni, old[iend - 1]);
            KT v[U][V];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ib = i0 + (u * 32 + lane) * V;
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
                if (ib < n) q = __ldg(reinterpret_cast<const uint4 *>(old + ib));
                memcpy(v[u], &q, 16);
            }
            int dbefore[U][V], ibefore[U][V];
            bool gone[U][V];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    dbefore[u][e] = d_lo;
                    ibefore[u][e] = i_lo;
                    gone[u][e] = false;
                }
            for (int b = d_lo; b < d_hi; b += 32) {
                const int pl = b + lane < d_hi ? DP[b + lane] : 0x7fffffff;
                const int m = min(32, d_hi - b);
                for (int k = 0; k < m; ++k) {
                    const int pk = __shfl_sync(0xffffffffu, pl, k);
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const int i = i0 + (u * 32 + lane) * V + e;
                            dbefore[u][e] += pk < i;
                            gone[u][e] |= pk == i;
                        }
                }
            }
            for (int b = i_lo; b < i_hi; b += 32) {
                const KT ul = b + lane < i_hi ? I[b + lane] : KT(0);
                const int m = min(32, i_hi - b);
                for (int k = 0; k < m; ++k) {
                    const KT uk = shfl_key(ul, k);
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int e = 0; e < V; ++e) ibefore[u][e] += !(v[u][e] < uk);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const int i = i0 + (u * 32 + lane) * V + e;
                    if (i < n && !gone[u][e]) {
                        const int pos = i - dbefore[u][e] + ibefore[u][e];
                        if (pos < 0 || pos >= nn) flag_error(status);
                        else dst[pos] = v[u][e];
                    }
                }
        }
        // insert j lands at j + #(old < u_j) - #(deletes < u_j)
        for (int j = lane; j < ni; j += 32) {
            const KT u = I[j];
            const int pos = j + IL[j] - lower_bound_k<KT>(Dl, nd, u);
            if (pos < 0 || pos >= nn) flag_error(status);
            else dst[pos] = u;
        }
    }
}


// Lanes per bin of the light merge (two bins per warp: the per-bin work of
// reading the bin's sizes and offsets and indexing its new run is shared by
// two bins, and 16 lanes x 8 keys cover the few hundred keys of a bin in one
// or a few passes).
constexpr int kMergeLanes = 16;

// What a light merge reads about its bin before touching keys.
struct LightBin {
    uint32_t ni, nd;    // inserts, deletes
    uint32_t ooff, on;  // old run: first node, keys
    uint32_t noff, nn;  // new run
    uint32_t io, dof;   // first insert, first delete
};

__device__ __forceinline__ LightBin light_bin_load(const BinHdr *old_hdr, const BinHdr *new_hdr,
                                                   const uint32_t *ins_off, const uint32_t *ins_n,
                                                   const uint32_t *del_off, const uint32_t *del_n, int64_t g)
{
    LightBin b;
    b.ni = ins_n[g];
    b.nd = del_n[g];
    const uint2 o = *reinterpret_cast<const uint2 *>(old_hdr + g), w = *reinterpret_cast<const uint2 *>(new_hdr + g);
    b.ooff = o.x;
    b.on = bin_count(o.y);
    b.noff = w.x;
    b.nn = bin_count(w.y);
    b.io = ins_off[g];
    b.dof = del_off[g];
    return b;
}

// Merge of a bin with at most 32 inserts and at most 32 deletes (nearly
// every bin of an update), in the old run's index space only: insert j
// precedes old key i iff its lower bound lb_j <= i, delete k removes old key
// pos_k, so a kept old key i lands at i + #(lb_j <= i) - #(pos_k < i) and
// insert j at lb_j + (its rank among the inserts) - #(pos_k < lb_j).  W
// lanes of a warp serve the bin (lane = 0..W-1 among them, mask = their
// bits); lane L holds old keys i0 + L + W e (e < 8), so that the loads and
// stores of the lanes touch consecutive keys.  Each delta adds one to a byte
// counter of the first e it covers, and one multiply by 0x0101..01 turns the
// eight byte counters into their prefix sums (at most 32 per byte, no
// carries).  The deltas are read W at a time and broadcast by shuffles.
template <typename KT, int W>
__device__ __forceinline__ void merge_bin_light(const void *old_store, void *new_store, const KT *ins_keys,
                                                const int32_t *ins_lb, const int32_t *del_pos, const LightBin &b,
                                                int lane, unsigned mask, int *status)
{
    const KT *old = leaf_run<KT>(const_cast<void *>(old_store), b.ooff, b.on);
    KT *dst = leaf_run<KT>(new_store, b.noff, b.nn);
    const int n = (int)b.on, ni = (int)b.ni, nd = (int)b.nd, nn = (int)b.nn;
    const uint32_t io = b.io, dof = b.dof;
    // Every delete must name a distinct old key (the locate pass flags one
    // that does not and gives it position 0x7fffffff) and the new size must
    // be n + ni - nd; then the positions below are a bijection onto [0, nn)
    // and need no further checks.  A bin that breaks this is flagged and
    // left unwritten.
    bool bad = nd > n || nn != n + ni - nd;
    for (int k0 = 0; k0 < nd; k0 += W)
        bad |= k0 + lane < nd && (uint32_t)del_pos[dof + k0 + lane] >= (uint32_t)n;
    if (__any_sync(mask, bad)) {
        if (lane == 0) flag_error(status);
        return;
    }
    if (ni == 0 && nd == 0) {
        constexpr int V = 16 / (int)sizeof(KT);  // whole 16-byte pieces lie inside the padded run
        for (int i = lane * V; i < n; i += W * V)
            *reinterpret_cast<uint4 *>(dst + i) = __ldg(reinterpret_cast<const uint4 *>(old + i));
        return;
    }
    constexpr int E = 8;
    constexpr unsigned long long kOnes = 0x0101010101010101ull;
    for (int i0 = 0; i0 < n; i0 += W * E) {
        const int base = i0 + lane;  // this lane's key e = 0
        const KT *src = old + base;
        KT v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = base + W * e < n ? src[W * e] : KT(0);
        // changes before this pass shift every key of it alike (a count in
        // byte 0); only those inside it are placed key slot by key slot
        const int iend = i0 + W * E;
        unsigned long long ih = 0, dh = 0;
        uint32_t gone = 0;
        for (int k0 = 0; k0 < ni; k0 += W) {
            const bool v = k0 + lane < ni;
            const int lb = v ? ins_lb[io + k0 + lane] : 0;
            ih += (unsigned)__popc(group_ballot<W>(mask, v && lb < i0));
            for (uint32_t in = group_ballot<W>(mask, v && lb >= i0 && lb < iend); in; in &= in - 1) {
                const int t = __shfl_sync(mask, lb, __ffs(in) - 1, W) - base;  // keys >= lb: e >= ceil(t / W)
                const int et = t <= 0 ? 0 : (t + W - 1) / W;
                if (et < E) ih += 1ull << (8 * et);
            }
        }
        for (int k0 = 0; k0 < nd; k0 += W) {
            const bool v = k0 + lane < nd;
            const int dp = v ? del_pos[dof + k0 + lane] : 0;
            dh += (unsigned)__popc(group_ballot<W>(mask, v && dp < i0));
            for (uint32_t in = group_ballot<W>(mask, v && dp >= i0 && dp < iend); in; in &= in - 1) {
                const int t = __shfl_sync(mask, dp, __ffs(in) - 1, W) - base;  // keys > pos: e >= ceil((t + 1) / W)
                const int et = t < 0 ? 0 : (t + W) / W;
                if (et < E) dh += 1ull << (8 * et);
                if (t >= 0 && t % W == 0 && t < W * E) gone |= 1u << (t / W);
            }
        }
        // byte e of sh: 64 + inserts before key e - deletes before it (each
        // prefix sum is at most 32, so no byte borrows from its neighbour)
        const unsigned long long sh = ih * kOnes + 0x4040404040404040ull - dh * kOnes;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (base + W * e < n && !((gone >> e) & 1u))
                dst[base + W * e + (int)((sh >> (8 * e)) & 0xffu) - 64] = v[e];
    }
    // inserts: lb + rank among the inserts (equal keys in index order) -
    // deletes below it; insert j is taken by lane j mod W
    for (int j0 = 0; j0 < ni; j0 += W) {
        const bool mine = j0 + lane < ni;
        const KT ik = mine ? ins_keys[io + j0 + lane] : KT(0);
        const int ilb = mine ? ins_lb[io + j0 + lane] : 0;
        int r = ilb;
        for (int k0 = 0; k0 < ni; k0 += W) {
            const KT uk_l = k0 + lane < ni ? ins_keys[io + k0 + lane] : KT(0);
            const int m = min(W, ni - k0);
            for (int k = 0; k < m; ++k) {
                const KT uk = shfl_key_w<W>(mask, uk_l, k);
                r += (uk < ik) || (uk == ik && k0 + k < j0 + lane);
            }
        }
        for (int k0 = 0; k0 < nd; k0 += W) {
            const int dp = k0 + lane < nd ? del_pos[dof + k0 + lane] : 0;
            const int m = min(W, nd - k0);
            for (int k = 0; k < m; ++k) r -= __shfl_sync(mask, dp, k, W) < ilb;
        }
        if (mine) dst[r] = ik;
    }
}

// A bin takes the light merge when it has at most 32 inserts and at most 32
// deletes (the segmented sort leaves exactly those delta lists unsorted).
__device__ __forceinline__ bool light_bin(uint32_t ni, uint32_t nd) { return ni <= 32 && nd <= 32; }

// W lanes per light bin (32 / W bins per warp): merge, then index the new
// run (its keys were just written by these lanes and are read back from L2,
// not HBM).  Heavy bins are listed for upd_merge_kernel.
template <typename KT, int W>
__global__ void __launch_bounds__(256, 5) upd_merge_light_kernel(const void *old_store, const BinHdr *old_hdr,
                                                                 void *new_store, BinHdr *new_hdr, const KT *ins_keys,
                                                                 const uint32_t *ins_off, const uint32_t *ins_n,
                                                                 const uint32_t *del_off, const uint32_t *del_n,
                                                                 const int32_t *ins_lb, const int32_t *del_pos,
                                                                 int64_t nbins, uint32_t *heavy, uint32_t *n_heavy,
                                                                 int *status)
{
    const int lane = threadIdx.x & (W - 1);
    const unsigned mask = W == 32 ? 0xffffffffu : ((1u << W) - 1u) << (threadIdx.x & 31 & ~(W - 1));
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) / W) {
        const LightBin b = light_bin_load(old_hdr, new_hdr, ins_off, ins_n, del_off, del_n, g);
        if (!light_bin(b.ni, b.nd)) {  // left to upd_merge_kernel
            if (lane == 0) heavy[atomicAdd(n_heavy, 1u)] = (uint32_t)g;
            continue;
        }
        merge_bin_light<KT, W>(old_store, new_store, ins_keys, ins_lb, del_pos, b, lane, mask, status);
        __syncwarp(mask);
        index_bin<KT, W>(new_store, new_hdr, g, lane, mask);
    }
}

// The other bins (more than 32 inserts or deletes; sorted delta lists), the
// n_heavy of them that upd_merge_light_kernel listed, one warp per bin,
// merged by merge_bin.
template <typename KT>
__global__ void __launch_bounds__(256, 4) upd_merge_kernel(const void *old_store, const BinHdr *old_hdr, void *new_store, BinHdr *new_hdr,
                                 const KT *ins_keys, const uint32_t *ins_off, const uint32_t *ins_n, const KT *del_keys,
                                 const uint32_t *del_off, const uint32_t *del_n, const int32_t *ins_lb,
                                 const int32_t *del_pos, const uint32_t *heavy, const uint32_t *n_heavy, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t nh = *n_heavy;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nh;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t g = heavy[t];
        merge_bin<KT>(old_store, old_hdr, new_store, new_hdr, ins_keys, ins_off, ins_n, del_keys, del_off, del_n,
                      ins_lb, del_pos, g, lane, status);
        __syncwarp();
        index_bin<KT>(new_store, new_hdr, g, lane);
    }
}

// Grow-only device buffer of the handle (freed with the handle).
static cddt_status reserve(void **buf, size_t *have, size_t bytes)
{
    if (bytes <= *have) return CDDT_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    const size_t want = bytes + bytes / 4;
    CDDT_CUDA(cudaMalloc(buf, want));
    *have = want;
    return CDDT_OK;
}

// Online update (Section IV-D, batched): all temporaries live in the
// handle's workspaces and the new store goes into the buffer the previous
// update left behind, so a steady stream of updates allocates nothing.
template <typename KT>
static cddt_status update_kt(cddt_s *h, const int32_t *xy, const uint8_t *occ, int32_t n, cudaStream_t st)
{
    const int64_t ncell = (int64_t)h->W * h->H;
    const int64_t nb = h->total_bins;
    if (!h->last_writer) {
        CDDT_CUDA(cudaMalloc(&h->last_writer, sizeof(int32_t) * (size_t)ncell));
        CDDT_CUDA(cudaMemsetAsync(h->last_writer, 0xff, sizeof(int32_t) * (size_t)ncell, st));
        CDDT_CUDA(cudaMalloc(&h->stamp, sizeof(uint32_t) * (size_t)ncell));
        CDDT_CUDA(cudaMemsetAsync(h->stamp, 0, sizeof(uint32_t) * (size_t)ncell, st));
        h->epoch = 0;
    }
    if (++h->epoch == 0) {
        CDDT_CUDA(cudaMemsetAsync(h->stamp, 0, sizeof(uint32_t) * (size_t)ncell, st));
        h->epoch = 1;
    }
    // workspace: every piece below, sized by n and the bin count
    const size_t sse = (size_t)scan_scratch_elems(nb);
    const size_t nbz = (size_t)std::max<int64_t>(nb, 1);
    size_t bytes = Arena::need(4 * (size_t)n) + Arena::need(36 * (size_t)n) + Arena::need(8) +
                   Arena::need(20 * nbz) + Arena::need(8 * sse) + Arena::need(16) + Arena::need(8 * nbz) +
                   Arena::need(sizeof(BinHdr) * nbz) + 2 * (Arena::need(4 * 8 * nbz) + Arena::need(4 * 8)) +
                   Arena::need(4 * nbz) + 2 * Arena::need(8 * sse) + Arena::need(24) + Arena::need(4 * nbz) +
                   Arena::need(16);
    CDDT_TRY(reserve(&h->ws, &h->ws_bytes, bytes));
    Arena ws{reinterpret_cast<char *>(h->ws), h->ws_bytes, 0};
    uint32_t *changed = ws.take<uint32_t>((size_t)n), *flips = ws.take<uint32_t>(9 * (size_t)n);
    uint32_t *nchanged = ws.take<uint32_t>(2), *nflips = nchanged + 1;
    uint32_t *arr = ws.take<uint32_t>(5 * nbz);
    uint64_t *scratch = ws.take<uint64_t>(sse), *tot = ws.take<uint64_t>(2);
    uint32_t *cur = ws.take<uint32_t>(2 * nbz);
    BinHdr *old_hdr = ws.take<BinHdr>(nbz);
    uint32_t *heavy = ws.take<uint32_t>(nbz), *n_heavy = ws.take<uint32_t>(4);
    if (!changed || !flips || !nchanged || !arr || !scratch || !tot || !cur || !old_hdr || !heavy || !n_heavy)
        return CDDT_ERR_OOM;
    CDDT_CUDA(cudaMemsetAsync(nchanged, 0, sizeof(uint32_t) * 2, st));
    const unsigned gn = grid_cap(n, 256);
    upd_dedupe_kernel<<<gn, 256, 0, st>>>(xy, n, h->W, h->H, h->last_writer, h->status);
    upd_apply_kernel<<<gn, 256, 0, st>>>(xy, occ, n, h->W, h->H, h->last_writer, h->grid, changed, nchanged);
    upd_flip_kernel<<<gn, 256, 0, st>>>(changed, nchanged, h->W, h->H, h->grid, h->edge, h->stamp, h->epoch, flips,
                                        nflips);
    // per-bin insert / delete counts and offsets
    uint32_t *ins_n = arr, *del_n = ins_n + nb, *ins_off = del_n + nb, *del_off = ins_off + nb, *new_n = del_off + nb;
    CDDT_CUDA(cudaMemsetAsync(ins_n, 0, sizeof(uint32_t) * 2 * (size_t)nb, st));
    const unsigned gd = grid_cap((int64_t)9 * n * h->S, 256, 32);
    upd_delta_kernel<KT, 0><<<gd, 256, 0, st>>>(flips, nflips, h->W, h->slices, h->S, h->Q, ins_n, del_n, nullptr,
                                                nullptr, nullptr, nullptr, nullptr, nullptr);
    exclusive_scan_u32(ins_n, ins_off, nb, scratch, tot, st);
    exclusive_scan_u32(del_n, del_off, nb, scratch, tot + 1, st);
    upd_newcount_kernel<<<grid_cap(nb, 256), 256, 0, st>>>(h->hdr, ins_n, del_n, nb, new_n, h->status);
    uint64_t totals[2];
    CDDT_CUDA(cudaMemcpyAsync(totals, tot, sizeof(totals), cudaMemcpyDeviceToHost, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    CDDT_CUDA(cudaGetLastError());
    if (totals[0] + totals[1] == 0) return CDDT_OK;  // no edge status changed
    // per delta: key, bin and (after the sort) its place in the old bin
    const size_t ni_t = (size_t)std::max<uint64_t>(totals[0], 1), nd_t = (size_t)std::max<uint64_t>(totals[1], 1);
    const size_t kb = Arena::need(sizeof(KT) * ni_t) + Arena::need(sizeof(KT) * nd_t) + Arena::need(4 * ni_t) +
                      Arena::need(4 * nd_t) + Arena::need(4 * ni_t) + Arena::need(4 * nd_t);
    CDDT_TRY(reserve(&h->ws_keys, &h->ws_keys_bytes, kb));
    Arena wk{reinterpret_cast<char *>(h->ws_keys), h->ws_keys_bytes, 0};
    KT *ins_keys = wk.take<KT>(ni_t), *del_keys = wk.take<KT>(nd_t);
    uint32_t *ins_bin = wk.take<uint32_t>(ni_t), *del_bin = wk.take<uint32_t>(nd_t);
    int32_t *ins_lb = wk.take<int32_t>(ni_t), *del_pos = wk.take<int32_t>(nd_t);
    uint32_t *ins_cur = cur, *del_cur = cur + nb;
    CDDT_CUDA(cudaMemsetAsync(cur, 0, sizeof(uint32_t) * 2 * (size_t)nb, st));
    upd_delta_kernel<KT, 1><<<gd, 256, 0, st>>>(flips, nflips, h->W, h->slices, h->S, h->Q, ins_cur, del_cur, ins_off,
                                                del_off, ins_keys, del_keys, ins_bin, del_bin);
    // only bins with more than 32 inserts or deletes need sorted lists (the
    // merge's binary-search path); the others are merged in any order
    cddt_status rc =
        sort_segments<KT>(Segs<KT>{nullptr, nullptr, ins_keys, ins_off, ins_n, del_n, 32}, nb, st, &ws);
    if (rc == CDDT_OK)
        rc = sort_segments<KT>(Segs<KT>{nullptr, nullptr, del_keys, del_off, del_n, ins_n, 32}, nb, st, &ws);
    if (rc != CDDT_OK) return rc;
    // places of the deltas in the old store, a new layout into the spare
    // store, then the merge from the old store
    CDDT_CUDA(cudaMemcpyAsync(old_hdr, h->hdr, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st));
    if (totals[0])
        upd_locate_kernel<KT><<<grid_cap((int64_t)totals[0], 256), 256, 0, st>>>(
            ins_keys, ins_bin, ins_off, ins_n, del_n, (int64_t)totals[0], false, h->store, old_hdr, ins_lb, h->status);
    if (totals[1])
        upd_locate_kernel<KT><<<grid_cap((int64_t)totals[1], 256), 256, 0, st>>>(
            del_keys, del_bin, del_off, del_n, ins_n, (int64_t)totals[1], true, h->store, old_hdr, del_pos, h->status);
    void *store = nullptr;
    int64_t nodes = 0;
    rc = layout_bins(h, new_n, st, &store, &nodes, std::max<int64_t>(h->store_nodes / 8, 1024), &ws, &h->spare,
                     &h->spare_nodes);
    if (rc != CDDT_OK) {
        cudaMemcpyAsync(h->hdr, old_hdr, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
        return rc;
    }
    const int64_t store_cap = h->spare_nodes;
    CDDT_CUDA(cudaMemsetAsync(n_heavy, 0, sizeof(uint32_t), st));
    upd_merge_light_kernel<KT, kMergeLanes><<<grid_cap(nb * kMergeLanes, 256), 256, 0, st>>>(
        h->store, old_hdr, store, h->hdr, ins_keys, ins_off, ins_n, del_off, del_n, ins_lb, del_pos, nb, heavy, n_heavy,
        h->status);
    upd_merge_kernel<KT><<<sm_count() * 4, 256, 0, st>>>(h->store, old_hdr, store, h->hdr, ins_keys, ins_off, ins_n,
                                                        del_keys, del_off, del_n, ins_lb, del_pos, heavy, n_heavy,
                                                        h->status);
    CDDT_CUDA(cudaGetLastError());
    // the old store becomes the next update's target (stream order keeps the
    // merge's reads of it before any later write)
    h->spare = h->store;
    h->spare_nodes = h->store_cap;
    h->store = store;
    h->store_nodes = nodes;
    h->store_cap = store_cap;
    return CDDT_OK;
}

cddt_status update_cells(cddt_s *h, const int32_t *xy, const uint8_t *occ, int32_t n, cudaStream_t st)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    cddt_status rc = h->u16 ? update_kt<uint16_t>(h, xy, occ, n, st) : update_kt<float>(h, xy, occ, n, st);
    if (rc == CDDT_OK) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&h->update_ms, e0, e1);
    }
    h->generation++;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace cddt
