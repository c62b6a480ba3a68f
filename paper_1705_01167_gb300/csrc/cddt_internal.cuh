// cddt_internal.cuh -- device data layout and device functions of the GB300
// CDDT library.  Shared by the translation units of libcddt.so only.
//
// Layout of one CDDT in HBM
// -------------------------
//  slices  SliceInfo[S]  (S = N/2 stored slices, Section IV-C): cos, sin of
//          theta_s = 2 pi s / N, the integer bin offset T_s, the bin count,
//          the first global bin of the slice and the 16-bit offset X_s.
//  bins    uint2[total_bins]: {node offset in 32-byte nodes, zero-point count n}.
//  store   32-byte nodes.  Each bin owns a contiguous, 32-byte aligned run of
//          nodes: the internal nodes of an implicit K-ary search tree (root
//          first, then each level down) followed by its ceil(n/K) leaf nodes,
//          which hold the bin's zero points sorted ascending, padded with +inf
//          (K = 8 float32 keys, or 16 uint16 keys per node).  Separator c of an
//          internal node at level l is the largest key of its child's subtree
//          (child j covers keys [j K^l, (j+1) K^l)).  A search reads one node
//          per level: the root and upper levels are small and stay in L2, the
//          leaf is one sector.
//  grid    uint8[H][W] occupancy (nonzero = occupied), edge uint8[H][W].
//
// Float contract: every float32 step of the projection, binning and range is
// an explicitly rounded intrinsic (__fmul_rn, __fadd_rn, __fsub_rn), which the
// compiler never fuses, in the order the readings of the paper fix.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cddt.h"

namespace cddt {

constexpr float kInf = __builtin_huge_valf();

struct __align__(16) SliceInfo {
    float c, s;      // cos, sin of theta_s
    int32_t T;       // integer bin offset
    int32_t nb;      // bins in the slice
    uint32_t sbase;  // first global bin
    float X;         // 16-bit key offset (integer-valued)
    int32_t pad0, pad1;
};

// Everything a query kernel needs to read one CDDT.
struct MapView {
    const SliceInfo *slices;
    const uint2 *bins;
    const void *store;
    const uint8_t *grid;
    int32_t W, H, N, S;
    float max_range;
    float inv_step;  // (float)(N / (2 pi)), computed in double
    float Q, invQ;   // 16-bit scale and its inverse (powers of two)
    int32_t u16;
    int32_t search;  // CDDT_SEARCH_*
};

// ------------------------------------------------------------ geometry

// Discrete direction of a query (reading S1): k = round-half-up(theta N / 2pi)
// wrapped into [0, N).  Returns false for a non-finite theta.
__device__ __forceinline__ bool query_dir(float theta, float inv_step, int N, int &k)
{
    float t = __fmul_rn(theta, inv_step);
    float tk = floorf(__fadd_rn(t, 0.5f));
    if (fabsf(tk) < 16777216.0f) {
        int ki = (int)tk % N;
        k = ki < 0 ? ki + N : ki;
        return true;
    }
    if (!isfinite(tk)) return false;
    int ki = (int)fmodf(tk, (float)N);
    k = ki < 0 ? ki + N : ki;
    return true;
}

// Occupancy pre-check (Section IV-C): the query may be cast only from a free,
// in-map cell.
__device__ __forceinline__ bool free_cell(const uint8_t *grid, int W, int H, float x, float y)
{
    float fx = floorf(__fadd_rn(x, 0.5f));
    float fy = floorf(__fadd_rn(y, 0.5f));
    if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) return false;
    return __ldg(grid + (int64_t)(int)fy * W + (int)fx) == 0;
}

// Edge status of cell (i, j) (Section IV-A: map minus its 3x3 erosion; an
// occupied cell with a free or off-map 8-neighbour).
__device__ __forceinline__ uint8_t edge_at(const uint8_t *g, int W, int H, int i, int j)
{
    if (!g[(int64_t)j * W + i]) return 0;
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            if (!di && !dj) continue;
            int a = i + di, b = j + dj;
            if (a < 0 || a >= W || b < 0 || b >= H) return 1;
            if (!g[(int64_t)b * W + a]) return 1;
        }
    return 0;
}

// Projection P_DDT (reading S3): xr = x c + y s, yr = y c - x s.
__device__ __forceinline__ void project(float x, float y, float c, float s, float &xr, float &yr)
{
    xr = __fadd_rn(__fmul_rn(x, c), __fmul_rn(y, s));
    yr = __fsub_rn(__fmul_rn(y, c), __fmul_rn(x, s));
}

__device__ __forceinline__ int query_bin(float yr, int T)
{
    return (int)floorf(__fadd_rn(yr, 0.5f)) + T;
}

__device__ __forceinline__ float half_extent(float c, float s)
{
    return __fmul_rn(0.5f, __fadd_rn(fabsf(c), fabsf(s)));
}

// Bins whose open interval meets the open y'-extent of a cell (reading S4).
__device__ __forceinline__ bool cell_bins(float yr, float h, int T, int nb, int &b0, int &b1)
{
    float lo = __fsub_rn(__fsub_rn(yr, h), 0.5f);
    float hi = __fadd_rn(__fadd_rn(yr, h), 0.5f);
    int a = (int)floorf(lo) + 1 + T;
    int b = (int)ceilf(hi) - 1 + T;
    a = a < 0 ? 0 : a;
    b = b > nb - 1 ? nb - 1 : b;
    b0 = a;
    b1 = b;
    return a <= b;
}

// 16-bit key of a projected abscissa (reading S7) and its exact value.
__device__ __forceinline__ uint16_t quantise(float xr, float X, float Q)
{
    float w = floorf(__fadd_rn(__fmul_rn(__fadd_rn(xr, X), Q), 0.5f));
    w = fminf(fmaxf(w, 0.0f), 65535.0f);
    return (uint16_t)w;
}
__device__ __forceinline__ float dequantise(uint32_t key, float X, float invQ)
{
    return __fsub_rn(__fmul_rn((float)key, invQ), X);
}

// ------------------------------------------------------------ bin layout

// log2 of keys per 32-byte node.
template <typename KT> struct KeyT;
template <> struct KeyT<float> {
    static constexpr int LK = 3;
    static constexpr int K = 8;
};
template <> struct KeyT<uint16_t> {
    static constexpr int LK = 4;
    static constexpr int K = 16;
};

__host__ __device__ __forceinline__ int tree_levels(uint32_t L0, int LK)
{
    if (L0 <= 1) return 0;
    uint32_t v = L0 - 1;
    int bits = 0;
    while (v) { ++bits; v >>= 1; }
    return (bits + LK - 1) / LK;
}

// Nodes of a bin of n keys: internal nodes above ceil(n/K) leaves.
__host__ __device__ __forceinline__ uint32_t internal_nodes(uint32_t n, int LK)
{
    if (n == 0) return 0;
    uint32_t L0 = ((n - 1) >> LK) + 1;
    int h = tree_levels(L0, LK);
    uint32_t t = 0;
    for (int l = 1; l <= h; ++l) t += ((L0 - 1) >> (LK * l)) + 1;
    return t;
}
__host__ __device__ __forceinline__ uint32_t bin_nodes(uint32_t n, int LK)
{
    if (n == 0) return 0;
    return internal_nodes(n, LK) + ((n - 1) >> LK) + 1;
}

// A 32-byte node read as K keys, compared in float (reading S5 semantics).
struct NodeF {
    float v[8];
    __device__ __forceinline__ void load(const void *p)
    {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};

// Number of keys <= x (Upper) or < x (!Upper) in a node.
template <bool Upper>
__device__ __forceinline__ int count_node(const float *v, int K, float x)
{
    int c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c += Upper ? (v[i] <= x) : (v[i] < x);
    (void)K;
    return c;
}

__device__ __forceinline__ float pick8(const float *v, int i)
{
    float r = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) r = (i == k) ? v[k] : r;
    return r;
}

// ---------------------------------------------------------------- search

// Search result: index of the first key > x (Upper) or >= x (!Upper) in the
// bin, n when none; also the key at that index (when < n) and the key just
// before it (when the index is > 0), which the paired reverse beam uses.
struct SearchResult {
    int idx;
    float at;    // key[idx]
    float prev;  // key[idx - 1]
};

// Key i of a bin from the leaf run (scalar load, L1-resident after a search).
template <typename KT>
__device__ __forceinline__ float bin_key(const MapView &m, const uint2 &bi, uint32_t internal, int i,
                                         float X)
{
    if (sizeof(KT) == 4) {
        const float *leaf = reinterpret_cast<const float *>(m.store) + ((size_t)(bi.x + internal) << 3);
        return __ldg(leaf + i);
    } else {
        const uint16_t *leaf =
            reinterpret_cast<const uint16_t *>(m.store) + ((size_t)(bi.x + internal) << 4);
        return dequantise(__ldg(leaf + i), X, m.invQ);
    }
}

// Descend the implicit tree of one bin (layout above).
template <typename KT, bool Upper>
__device__ __forceinline__ SearchResult tree_search(const MapView &m, const uint2 &bi, float x, float X)
{
    constexpr int LK = KeyT<KT>::LK;
    constexpr int K = KeyT<KT>::K;
    SearchResult r;
    const uint32_t n = bi.y;
    r.idx = 0;
    r.at = kInf;
    r.prev = -kInf;
    if (n == 0) return r;
    const uint32_t L0 = ((n - 1) >> LK) + 1;
    const int h = tree_levels(L0, LK);
    const char *base = reinterpret_cast<const char *>(m.store) + ((size_t)bi.x << 5);
    uint32_t off = 0;  // node offset of the current level
    uint32_t k = 0;    // node index inside the level
    uint32_t internal = 0;
    for (int l = h; l >= 1; --l) internal += ((L0 - 1) >> (LK * l)) + 1;
    for (int l = h; l >= 1; --l) {
        int c = 0;
        if (sizeof(KT) == 4) {
            NodeF nd;
            nd.load(base + ((size_t)(off + k) << 5));
            c = count_node<Upper>(nd.v, K, x);
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(base + ((size_t)(off + k) << 5));
            uint4 a = __ldg(p), b = __ldg(p + 1);
            uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float lo = dequantise(w[q] & 0xffffu, X, m.invQ);
                float hi = dequantise(w[q] >> 16, X, m.invQ);
                c += Upper ? ((lo <= x) + (hi <= x)) : ((lo < x) + (hi < x));
            }
        }
        // The root has cnt[h-1] real children, its other separators are +inf
        // padding; when every real child's maximum is <= x (or < x) there is
        // no answer in the bin.  Below the root the parent's choice
        // guarantees a real child whose maximum exceeds x.
        if (l == h && c >= (int)(((L0 - 1) >> (LK * (h - 1))) + 1)) {
            r.idx = (int)n;
            r.prev = bin_key<KT>(m, bi, internal, (int)n - 1, X);
            return r;
        }
        off += ((L0 - 1) >> (LK * l)) + 1;
        k = k * K + c;
    }
    // leaf
    int c = 0;
    float at = kInf, prev = -kInf;
    if (sizeof(KT) == 4) {
        NodeF nd;
        nd.load(base + ((size_t)(off + k) << 5));
        c = count_node<Upper>(nd.v, K, x);
        at = pick8(nd.v, c < 8 ? c : 7);
        prev = pick8(nd.v, c > 0 ? c - 1 : 0);
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(base + ((size_t)(off + k) << 5));
        uint4 a = __ldg(p), b = __ldg(p + 1);
        uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        float vals[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            vals[2 * q] = dequantise(w[q] & 0xffffu, X, m.invQ);
            vals[2 * q + 1] = dequantise(w[q] >> 16, X, m.invQ);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) c += Upper ? (vals[q] <= x) : (vals[q] < x);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            at = (q == c) ? vals[q] : at;
            prev = (q == c - 1) ? vals[q] : prev;
        }
    }
    r.idx = (int)(k * K) + c;
    if (r.idx >= (int)n) {
        r.idx = (int)n;
        r.at = kInf;
    } else {
        r.at = at;
    }
    if (r.idx > 0) r.prev = (c > 0) ? prev : bin_key<KT>(m, bi, internal, r.idx - 1, X);
    return r;
}

// Branch-free binary search of the bin's sorted leaf run (same answers).
template <typename KT, bool Upper>
__device__ __forceinline__ SearchResult binary_search(const MapView &m, const uint2 &bi, float x,
                                                      float X)
{
    constexpr int LK = KeyT<KT>::LK;
    SearchResult r;
    const int n = (int)bi.y;
    r.idx = 0;
    r.at = kInf;
    r.prev = -kInf;
    if (n == 0) return r;
    const uint32_t internal = internal_nodes(bi.y, LK);
    int base = 0, len = n;
    while (len > 1) {
        int half = len >> 1;
        float v = bin_key<KT>(m, bi, internal, base + half - 1, X);
        base = (Upper ? (v <= x) : (v < x)) ? base + half : base;
        len -= half;
    }
    float v = bin_key<KT>(m, bi, internal, base, X);
    int idx = base + (Upper ? (v <= x) : (v < x));
    r.idx = idx;
    if (idx < n) r.at = (idx == base) ? v : bin_key<KT>(m, bi, internal, idx, X);
    if (idx > 0) r.prev = (idx - 1 == base) ? v : bin_key<KT>(m, bi, internal, idx - 1, X);
    return r;
}

template <typename KT, bool Upper>
__device__ __forceinline__ SearchResult bin_search(const MapView &m, const uint2 &bi, float x, float X)
{
    if (m.search == CDDT_SEARCH_BINARY) return binary_search<KT, Upper>(m, bi, x, X);
    return tree_search<KT, Upper>(m, bi, x, X);
}

// ------------------------------------------------------------ one ray cast

// Result of casting one beam: range and its derivative direction.
struct Cast {
    float r;       // clamped range
    float dzx, dzy;  // d r / d(x, y): -(c, s) forward, +(c, s) backward, 0 if clamped / miss
    int kb;        // bin size searched (-1: none)
};

// Cast from an in-map free cell position (pre-check already passed) in
// direction k.  One search; if `pair` is set, the opposite direction k + N/2
// is answered from the same search (Section IV-C: index i - 1).
template <typename KT>
__device__ __forceinline__ void cast_pair(const MapView &m, float x, float y, int k, bool pair,
                                          Cast &fwd_out, Cast &bwd_out, bool &k_is_fwd)
{
    const int S = m.S;
    const bool bwd = k >= S;
    const int s = bwd ? k - S : k;
    k_is_fwd = !bwd;
    const float4 sa = __ldg(reinterpret_cast<const float4 *>(m.slices + s));
    const float4 sb = __ldg(reinterpret_cast<const float4 *>(m.slices + s) + 1);
    const float c = sa.x, sn = sa.y;
    const int T = __float_as_int(sa.z), nb = __float_as_int(sa.w);
    const uint32_t sbase = __float_as_uint(sb.x);
    const float X = sb.y;
    float xr, yr;
    project(x, y, c, sn, xr, yr);
    const int b = query_bin(yr, T);
    Cast f, r;
    f.r = r.r = m.max_range;
    f.dzx = f.dzy = r.dzx = r.dzy = 0.0f;
    f.kb = r.kb = -1;
    if (b >= 0 && b < nb) {
        const uint2 bi = __ldg(m.bins + sbase + b);
        f.kb = r.kb = (int)bi.y;
        if (!bwd || pair) {
            // forward: first key > x' (upper bound)
            SearchResult sr = bin_search<KT, true>(m, bi, xr, X);
            if (sr.idx < (int)bi.y) {
                float d = __fsub_rn(sr.at, xr);
                if (d < m.max_range) { f.r = d; f.dzx = -c; f.dzy = -sn; }
            }
            if (pair) {
                // backward from the same search: last key < x'
                float pv = sr.prev;
                int j = sr.idx - 1;
                if (j >= 0 && pv == xr) {
                    const uint32_t internal = internal_nodes(bi.y, KeyT<KT>::LK);
                    while (j >= 0 && pv == xr) {
                        --j;
                        if (j >= 0) pv = bin_key<KT>(m, bi, internal, j, X);
                    }
                }
                if (j >= 0) {
                    float d = __fsub_rn(xr, pv);
                    if (d < m.max_range) { r.r = d; r.dzx = c; r.dzy = sn; }
                }
            }
        } else {
            // backward only: last key < x' = (first key >= x') - 1
            SearchResult sr = bin_search<KT, false>(m, bi, xr, X);
            if (sr.idx > 0) {
                float d = __fsub_rn(xr, sr.prev);
                if (d < m.max_range) { r.r = d; r.dzx = c; r.dzy = sn; }
            }
        }
    }
    fwd_out = f;
    bwd_out = r;
}

// ------------------------------------------------------------ beam model

struct BeamConsts {
    float z_hit, z_short, z_max, z_rand;
    float inv_2s2, norm_hit, inv_s2, inv_sig;
    float lam, max_range, inv_max_range;
    int trunc;
};

inline BeamConsts make_beam_consts(const cddt_beam_model &m)
{
    BeamConsts b;
    b.z_hit = m.z_hit;
    b.z_short = m.z_short;
    b.z_max = m.z_max;
    b.z_rand = m.z_rand;
    double sig = m.sigma_hit;
    b.inv_2s2 = (float)(1.0 / (2.0 * sig * sig));
    b.norm_hit = (float)(1.0 / (sig * 2.5066282746310002));
    b.inv_s2 = (float)(1.0 / (sig * sig));
    b.inv_sig = (float)(1.0 / sig);
    b.lam = m.lambda_short;
    b.max_range = m.max_range;
    b.inv_max_range = (float)(1.0 / (double)m.max_range);
    b.trunc = m.hit_truncnorm;
    return b;
}

// Per-beam terms that depend on the measurement only.
struct BeamObs {
    float z;      // measured range clamped to [0, max_range]
    float e_lz;   // lambda e^{-lambda z}
    float c_mr;   // z_max [z >= max] + z_rand [z < max] / max_range
};

__device__ __forceinline__ BeamObs beam_obs(const BeamConsts &m, float obs)
{
    BeamObs o;
    float z = fminf(fmaxf(obs, 0.0f), m.max_range);
    o.z = z;
    o.e_lz = m.lam * expf(-m.lam * z);
    o.c_mr = (z >= m.max_range) ? m.z_max : m.z_rand * m.inv_max_range;
    return o;
}

// log p(z | z*) and, when wanted, d log p / d z*.
template <bool Grad>
__device__ __forceinline__ float beam_logp(const BeamConsts &m, const BeamObs &o, float zs, float &dlogp)
{
    const float d = o.z - zs;
    float p_hit = m.norm_hit * expf(-(d * d) * m.inv_2s2);
    float dhit = 0.0f;
    if (m.trunc) {
        float a = (m.max_range - zs) * m.inv_sig;
        float b = -zs * m.inv_sig;
        float D = normcdff(a) - normcdff(b);
        p_hit = p_hit / D;
        if (Grad) {
            const float r2pi = 0.3989422804014327f;
            float dD = (r2pi * expf(-0.5f * b * b) - r2pi * expf(-0.5f * a * a)) * m.inv_sig;
            dhit = p_hit * (d * m.inv_s2 - dD / D);
        }
    } else if (Grad) {
        dhit = p_hit * d * m.inv_s2;
    }
    float p_short = 0.0f, dshort = 0.0f;
    if (zs > 0.0f && o.z <= zs) {
        float den = -expm1f(-m.lam * zs);
        p_short = o.e_lz / den;
        if (Grad && o.z < zs) {
            float e = expf(-m.lam * zs);
            dshort = -m.lam * o.e_lz * e / (den * den);
        }
    }
    const float p = m.z_hit * p_hit + m.z_short * p_short + o.c_mr;
    if (Grad) dlogp = (m.z_hit * dhit + m.z_short * dshort) / p;
    return logf(p);
}

}  // namespace cddt

// ---------------------------------------------------------------- handle

struct cddt_s {
    int device = 0;
    int32_t W = 0, H = 0, N = 0, S = 0;
    float max_range = 0;
    uint32_t flags = 0;
    int32_t u16 = 0;
    float Q = 1, invQ = 1;
    int32_t pruned = 0;
    int32_t search = CDDT_SEARCH_TREE;
    int64_t total_bins = 0;
    int64_t n_zp = 0;          // zero points (host copy, exact after each sync point)
    int64_t n_edge = 0;
    int64_t store_nodes = 0;   // nodes in use
    int64_t store_cap = 0;     // nodes allocated
    int64_t max_bin = 0;
    float build_ms = 0, prune_ms = 0, update_ms = 0;
    // device buffers owned by the handle
    cddt::SliceInfo *slices = nullptr;
    uint2 *bins = nullptr;
    void *store = nullptr;
    uint8_t *grid = nullptr;
    uint8_t *edge = nullptr;
    int *status = nullptr;      // device status word
    // update scratch (allocated on first update)
    int32_t *last_writer = nullptr;  // [W*H], -1 when free
    uint32_t *stamp = nullptr;       // [W*H] epoch claims
    uint32_t epoch = 0;
    // query sort scratch
    void *qscratch = nullptr;
    int64_t qscratch_bytes = 0;

    cddt::MapView view() const
    {
        cddt::MapView v;
        v.slices = slices;
        v.bins = bins;
        v.store = store;
        v.grid = grid;
        v.W = W;
        v.H = H;
        v.N = N;
        v.S = S;
        v.max_range = max_range;
        v.inv_step = (float)((double)N / (2.0 * 3.14159265358979323846));
        v.Q = Q;
        v.invQ = invQ;
        v.u16 = u16;
        v.search = search;
        return v;
    }
};

// Host helpers shared by the translation units.
namespace cddt {
cddt_status cuda_status(cudaError_t e);
// Build the sorted, tree-indexed store from per-bin key lists; implemented in
// cddt_build.cu and reused by prune and update.
cddt_status build_index(cddt_s *h, cudaStream_t st);
}  // namespace cddt

#define CDDT_CUDA(call)                                                       \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return cddt::cuda_status(e_);                  \
    } while (0)
