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

template <typename KT>
__global__ void prune_mark_kernel(MapView m, float eps, uint8_t *keep)
{
    constexpr int LK = KeyT<KT>::LK;
    const uint64_t pol = policy_evict_last();
    const int64_t cells = (int64_t)m.W * m.H;
    const int64_t total = cells * m.S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t / cells);
        const int64_t q = t - (int64_t)s * cells;
        if (__ldg(m.grid + q)) continue;
        const int j = (int)(q / m.W), i = (int)(q - (int64_t)j * m.W);
        const SliceInfo si = m.slices[s];
        float xr, yr;
        project((float)i, (float)j, si.c, si.s, xr, yr);
        const float h = half_extent(si.c, si.s);
        int b0, b1;
        if (s == 0) {
            b0 = b1 = j + si.T;
        } else {
            const float lo = __fsub_rn(__fsub_rn(yr, h), eps), hi = __fadd_rn(__fadd_rn(yr, h), eps);
            b0 = (int)ceilf(__fsub_rn(lo, 0.5f)) + si.T;
            b1 = (int)floorf(__fadd_rn(hi, 0.5f)) + si.T;
        }
        b0 = max(b0, 0);
        b1 = min(b1, si.nb - 1);
        const float xlo = __fsub_rn(__fsub_rn(xr, h), eps), xhi = __fadd_rn(__fadd_rn(xr, h), eps);
        for (int b = b0; b <= b1; ++b) {
            const uint32_t g = si.sbase + (uint32_t)b;
            const BinHdr bh = m.hdr[g];
            const uint32_t bn = bin_count(bh.nm);
            if (bn == 0) continue;
            int kb;
            const int l = bin_search<KT, false, CDDT_SEARCH_TREE>(m, g, xlo, si.X, pol, kb).idx;  // first key >= xlo
            const int u = bin_search<KT, true, CDDT_SEARCH_TREE>(m, g, xhi, si.X, pol, kb).idx;   // first key > xhi
            const int m0 = max(l - 1, 0), m1 = min(u, (int)bn - 1);
            uint8_t *kp = keep + (((size_t)bh.off + internal_nodes(bn, LK, KeyT<KT>::R)) << LK);
            for (int mm = m0; mm <= m1; ++mm) kp[mm] = 1;
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
    const int64_t work = (int64_t)h->W * h->H * h->S;
    prune_mark_kernel<KT><<<grid_cap(work, 256, 152 * 32), 256, 0, st>>>(h->view(), prune_eps(h->W, h->H),
                                                                          keep.as<uint8_t>());
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
                                 const uint32_t *del_off, KT *ins_keys, KT *del_keys)
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
                if (ins) ins_keys[ins_off[g] + atomicAdd(ins_n + g, 1u)] = key;
                else del_keys[del_off[g] + atomicAdd(del_n + g, 1u)] = key;
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

// Merge each bin's old sorted keys with its sorted inserts, dropping one
// occurrence per delete.  For an old key v at index i (first occurrence a):
// it is deleted iff i - a < (#deletes equal to v); a kept key lands at
// i - #(deletes <= v) + #(inserts <= v).  An insert u at index j lands at
// j + #(old < u) - #(deletes < u).  (Inserts precede equal old keys.)
template <typename KT>
__global__ void upd_merge_kernel(const void *old_store, const BinHdr *old_hdr, void *new_store, const BinHdr *new_hdr,
                                 const KT *ins_keys, const uint32_t *ins_off, const uint32_t *ins_n, const KT *del_keys,
                                 const uint32_t *del_off, const uint32_t *del_n, int64_t nbins, int *status)
{
    const int lane = threadIdx.x & 31;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nbins;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const BinHdr ob = old_hdr[g], nb = new_hdr[g];
        const uint32_t obn = bin_count(ob.nm), nbn = bin_count(nb.nm);
        const KT *old = leaf_run<KT>(const_cast<void *>(old_store), ob.off, obn);
        KT *dst = leaf_run<KT>(new_store, nb.off, nbn);
        const int n = (int)obn, ni = (int)ins_n[g], nd = (int)min(del_n[g], obn), nn = (int)nbn;
        const KT *I = ins_keys + ins_off[g];
        const KT *Dl = del_keys + del_off[g];
        if (ni == 0 && nd == 0) {
            for (int i = lane; i < n && i < nn; i += 32) dst[i] = old[i];
            continue;
        }
        for (int i = lane; i < n; i += 32) {
            const KT v = old[i];
            const int a = lower_bound_k<KT>(old, n, v);
            const int r_lt = lower_bound_k<KT>(Dl, nd, v), r_le = upper_bound_k<KT>(Dl, nd, v);
            if (i - a < r_le - r_lt) continue;
            const int pos = i - r_le + upper_bound_k<KT>(I, ni, v);
            if (pos < 0 || pos >= nn) {
                flag_error(status);
                continue;
            }
            dst[pos] = v;
        }
        for (int j = lane; j < ni; j += 32) {
            const KT u = I[j];
            const int pos = j + lower_bound_k<KT>(old, n, u) - lower_bound_k<KT>(Dl, nd, u);
            if (pos < 0 || pos >= nn) {
                flag_error(status);
                continue;
            }
            dst[pos] = u;
        }
    }
}

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
    Buf changed, flips, counters;
    CDDT_CUDA(changed.alloc(sizeof(uint32_t) * (size_t)n));
    CDDT_CUDA(flips.alloc(sizeof(uint32_t) * 9 * (size_t)n));
    CDDT_CUDA(counters.alloc(sizeof(uint32_t) * 2));
    CDDT_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(uint32_t) * 2, st));
    uint32_t *nchanged = counters.as<uint32_t>(), *nflips = nchanged + 1;
    const unsigned gn = grid_cap(n, 256);
    upd_dedupe_kernel<<<gn, 256, 0, st>>>(xy, n, h->W, h->H, h->last_writer, h->status);
    upd_apply_kernel<<<gn, 256, 0, st>>>(xy, occ, n, h->W, h->H, h->last_writer, h->grid, changed.as<uint32_t>(), nchanged);
    upd_flip_kernel<<<gn, 256, 0, st>>>(changed.as<uint32_t>(), nchanged, h->W, h->H, h->grid, h->edge, h->stamp,
                                        h->epoch, flips.as<uint32_t>(), nflips);
    // per-bin insert / delete counts and offsets
    Buf arr, scratch, tot;
    CDDT_CUDA(arr.alloc(sizeof(uint32_t) * 5 * (size_t)std::max<int64_t>(nb, 1)));
    CDDT_CUDA(scratch.alloc(sizeof(uint64_t) * (size_t)scan_scratch_elems(nb)));
    CDDT_CUDA(tot.alloc(sizeof(uint64_t) * 2));
    uint32_t *ins_n = arr.as<uint32_t>(), *del_n = ins_n + nb, *ins_off = del_n + nb, *del_off = ins_off + nb,
             *new_n = del_off + nb;
    CDDT_CUDA(cudaMemsetAsync(ins_n, 0, sizeof(uint32_t) * 2 * (size_t)nb, st));
    const unsigned gd = grid_cap((int64_t)9 * n * h->S, 256, 152 * 32);
    upd_delta_kernel<KT, 0><<<gd, 256, 0, st>>>(flips.as<uint32_t>(), nflips, h->W, h->slices, h->S, h->Q, ins_n, del_n,
                                                nullptr, nullptr, nullptr, nullptr);
    exclusive_scan_u32(ins_n, ins_off, nb, scratch.as<uint64_t>(), tot.as<uint64_t>(), st);
    exclusive_scan_u32(del_n, del_off, nb, scratch.as<uint64_t>(), tot.as<uint64_t>() + 1, st);
    upd_newcount_kernel<<<grid_cap(nb, 256), 256, 0, st>>>(h->hdr, ins_n, del_n, nb, new_n, h->status);
    uint64_t totals[2];
    CDDT_CUDA(cudaMemcpyAsync(totals, tot.p, sizeof(totals), cudaMemcpyDeviceToHost, st));
    CDDT_CUDA(cudaStreamSynchronize(st));
    CDDT_CUDA(cudaGetLastError());
    if (totals[0] + totals[1] == 0) return CDDT_OK;  // no edge status changed
    Buf ins_keys, del_keys, cur;
    CDDT_CUDA(ins_keys.alloc(sizeof(KT) * (size_t)std::max<uint64_t>(totals[0], 1)));
    CDDT_CUDA(del_keys.alloc(sizeof(KT) * (size_t)std::max<uint64_t>(totals[1], 1)));
    CDDT_CUDA(cur.alloc(sizeof(uint32_t) * 2 * (size_t)nb));
    uint32_t *ins_cur = cur.as<uint32_t>(), *del_cur = ins_cur + nb;
    CDDT_CUDA(cudaMemsetAsync(cur.p, 0, sizeof(uint32_t) * 2 * (size_t)nb, st));
    upd_delta_kernel<KT, 1><<<gd, 256, 0, st>>>(flips.as<uint32_t>(), nflips, h->W, h->slices, h->S, h->Q, ins_cur, del_cur,
                                                ins_off, del_off, ins_keys.as<KT>(), del_keys.as<KT>());
    cddt_status rc = sort_segments<KT>(Segs<KT>{nullptr, nullptr, ins_keys.as<KT>(), ins_off, ins_n}, nb, st);
    if (rc == CDDT_OK) rc = sort_segments<KT>(Segs<KT>{nullptr, nullptr, del_keys.as<KT>(), del_off, del_n}, nb, st);
    if (rc != CDDT_OK) return rc;
    // new layout, then the merge from the old store into the new one
    Buf old_hdr;
    CDDT_CUDA(old_hdr.alloc(sizeof(BinHdr) * (size_t)nb));
    CDDT_CUDA(cudaMemcpyAsync(old_hdr.p, h->hdr, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st));
    void *store = nullptr;
    int64_t nodes = 0;
    rc = layout_bins(h, new_n, st, &store, &nodes, 0);
    if (rc != CDDT_OK) {
        cudaMemcpyAsync(h->hdr, old_hdr.p, sizeof(BinHdr) * nb, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
        return rc;
    }
    upd_merge_kernel<KT><<<grid_cap(nb * 32, 256), 256, 0, st>>>(h->store, old_hdr.as<BinHdr>(), store, h->hdr, ins_keys.as<KT>(),
                                                                 ins_off, ins_n, del_keys.as<KT>(), del_off, del_n, nb,
                                                                 h->status);
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
