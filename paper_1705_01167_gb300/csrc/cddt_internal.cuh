// cddt_internal.cuh -- device data layout and device functions of the GB300
// CDDT library.  Shared by the translation units of libcddt.so only.
//
// Layout of one CDDT in HBM
// -------------------------
//  slices  SliceInfo[S]  (S = N/2 stored slices, Section IV-C): cos, sin of
//          theta_s = 2 pi s / N, the integer bin offset T_s, the bin count,
//          the first global bin of the slice and the 16-bit offset X_s.
//  hdr     BinHdr[total_bins], 32 bytes each: the node offset of the bin's
//          run, its zero-point count n and the R separators of the root of
//          the bin's search tree (R = 6 float32 or 12 uint16 keys).  A bin of
//          at most R keys keeps the keys themselves in the header.
//  store   32-byte nodes.  Each bin owns a contiguous, 32-byte aligned run:
//          the internal levels of an implicit K-ary search tree (top level
//          first) followed by its ceil(n/K) leaf nodes, which hold the bin's
//          zero points sorted ascending, padded with +inf (K = 8 float32 or
//          16 uint16 keys per node).  The root (in the header) covers at most
//          R nodes of the top level.  Separator q of a node is the largest key
//          of its q-th child's subtree.  A search reads the header, one node
//          per internal level and one leaf: 3 sectors for the few-hundred-key
//          bins of a 2000 x 2000 corridor map.  Headers and internal nodes
//          are read with an L2 evict-last policy and leaves with an
//          evict-first one, so that the stream of leaf reads does not push
//          the upper levels out of L2.
//  grid    uint8[H][W] occupancy (nonzero = occupied), edge uint8[H][W].
//
// Float contract: every float32 step of the projection, binning and range is
// an explicitly rounded intrinsic (__fmul_rn, __fadd_rn, __fsub_rn), which the
// compiler never fuses, in the order the readings of the paper fix.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>
#include <cstring>

#include "../../include/cddt.h"

namespace cddt {

constexpr float kInf = __builtin_huge_valf();

// The first 16 bytes hold what a float32 query reads (one 16-byte load); a
// 16-bit query reads all 32 (one 32-byte load).
struct __align__(32) SliceInfo {
    float c, s;      // cos, sin of theta_s
    uint32_t sbase;  // first global bin
    uint32_t Tnb;    // T | nb << 16 (both < 65536)
    float X;         // 16-bit key offset (integer-valued)
    int32_t T;       // integer bin offset
    int32_t nb;      // bins in the slice
    int32_t pad;
};

// Everything a query kernel needs to read one CDDT.
// Per-bin header (see the layout above).
struct __align__(32) BinHdr {
    uint32_t off;   // first node of the bin's run
    uint32_t nm;    // zero points n (bits 0-23); once indexed also the stored
                    // levels h (bits 24-27) and the root's child count (28-31)
    uint32_t w[6];  // root separators, or the keys themselves when n <= R
};

constexpr uint32_t kMaxBinKeys = (1u << 24) - 1;
__host__ __device__ __forceinline__ uint32_t bin_count(uint32_t nm) { return nm & 0xffffffu; }

// A CDDT_CHECKED build checks every gather from the slice table, the bin
// headers and the store against its buffer (chk below).
#ifndef CDDT_CHECKED
#define CDDT_CHECKED 0
#endif

struct MapView {
    const SliceInfo *slices;
    const BinHdr *hdr;
    const void *store;
    const uint8_t *grid;
    int32_t W, H, N, S;
    float max_range;
    float inv_step;  // (float)(N / (2 pi)), computed in double
    float Q, invQ;   // 16-bit scale and its inverse (powers of two)
    int32_t u16;
    int32_t search;  // CDDT_SEARCH_*
#if CDDT_CHECKED
    int64_t hdr_bytes, store_bytes;  // extents of hdr and store
    int *status;                     // the handle's device status word
#endif
};

#if CDDT_CHECKED
static __device__ __align__(32) uint32_t chk_dummy[8];
#endif

// Bounds check of a gather (CDDT_CHECKED builds; elsewhere it returns p): an
// access of `bytes` at p outside [base, base + extent) records
// CDDT_ERR_BOUNDS in the handle's status word and reads a zeroed 32-byte
// dummy instead, so the kernel runs to its end without touching memory it
// does not own, and the host learns of it from cddt_get_status.
template <typename T>
__device__ __forceinline__ const T *chk(const MapView &m, const T *p, int bytes, const void *base, int64_t extent)
{
#if CDDT_CHECKED
    const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(base);
    if (a < b || a + (uintptr_t)bytes > b + (uintptr_t)extent) {
        atomicCAS(m.status, 0, (int)CDDT_ERR_BOUNDS);
        return reinterpret_cast<const T *>(chk_dummy);
    }
#else
    (void)m; (void)bytes; (void)base; (void)extent;
#endif
    return p;
}
template <typename T>
__device__ __forceinline__ const T *chk_store(const MapView &m, const T *p, int bytes)
{
#if CDDT_CHECKED
    return chk(m, p, bytes, m.store, m.store_bytes);
#else
    (void)m; (void)bytes;
    return p;
#endif
}
template <typename T>
__device__ __forceinline__ const T *chk_hdr(const MapView &m, const T *p, int bytes)
{
#if CDDT_CHECKED
    return chk(m, p, bytes, m.hdr, m.hdr_bytes);
#else
    (void)m; (void)bytes;
    return p;
#endif
}
template <typename T>
__device__ __forceinline__ const T *chk_slice(const MapView &m, const T *p, int bytes)
{
#if CDDT_CHECKED
    return chk(m, p, bytes, m.slices, (int64_t)m.S * (int64_t)sizeof(SliceInfo));
#else
    (void)m; (void)bytes;
    return p;
#endif
}

// ------------------------------------------------------------ geometry

// Direction of a continuous heading for the baseline casters (reading D1):
// cos and sin of theta in float32 by a fixed sequence of correctly rounded
// operations, reproducible bit for bit on any IEEE host.  A heading beyond
// 2^16 rad is first taken modulo the float nearest 2 pi (fmodf, exact); the
// nearest multiple j of pi/2 is removed in three parts (Cody & Waite's
// additive reduction, each part a fused multiply-add), which leaves r within
// [-pi/4, pi/4]; sin r and cos r are the Taylor polynomials to r^9 and r^10
// in Horner form; j mod 4 picks the quadrant.  Within 2 ulp and 1.2e-7 of
// the exact values (measured over random headings).  theta must be finite.
__device__ __forceinline__ void dir_sincos(float th, float &s, float &c)
{
    if (fabsf(th) > 65536.0f) th = fmodf(th, 0x1.921fb6p+2f);
    const float j = rintf(__fmul_rn(th, 0x1.45f306p-1f));
    float r = __fmaf_rn(-j, 0x1.921fb6p+0f, th);
    r = __fmaf_rn(-j, -0x1.777a5cp-25f, r);
    r = __fmaf_rn(-j, -0x1.ee59dap-50f, r);
    const float r2 = __fmul_rn(r, r);
    float ps = __fmaf_rn(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = __fmaf_rn(r2, ps, 1.0f / 120.0f);
    ps = __fmaf_rn(r2, ps, -1.0f / 6.0f);
    const float sn = __fmaf_rn(__fmul_rn(r2, r), ps, r);
    float pc = __fmaf_rn(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = __fmaf_rn(r2, pc, -1.0f / 720.0f);
    pc = __fmaf_rn(r2, pc, 1.0f / 24.0f);
    pc = __fmaf_rn(r2, pc, -0.5f);
    const float cs = __fmaf_rn(r2, pc, 1.0f);
    const int q = (int)j & 3;
    s = q == 0 ? sn : q == 1 ? cs : q == 2 ? -sn : -cs;
    c = q == 0 ? cs : q == 1 ? -sn : q == 2 ? -cs : sn;
}

// Discrete direction of a query (reading S1): k = round-half-up(theta N / 2pi)
// wrapped into [0, N).  Returns false for a non-finite theta.
__device__ __forceinline__ bool query_dir(float theta, float inv_step, int N, int &k)
{
    float t = __fmul_rn(theta, inv_step);
    const float th = __fadd_rn(t, 0.5f);
    // floor and convert in one step; within one turn either way of [0, N)
    // (an in-range heading plus a beam offset) one add or subtract of N wraps
    // it.  NaN converts to 0, so it is caught first.
    // Out-of-range values saturate and fall through to the general wrap.
    int kw = __float2int_rd(th);
    kw += kw < 0 ? N : 0;
    kw -= kw >= N ? N : 0;
    if ((unsigned)kw < (unsigned)N && th == th) {
        k = kw;
        return true;
    }
    const float tk = floorf(th);
    if (fabsf(tk) < 16777216.0f) {
        const int ki = (int)tk % N;
        k = ki < 0 ? ki + N : ki;
        return true;
    }
    if (!isfinite(tk)) return false;
    const int kf = (int)fmodf(tk, (float)N);
    k = kf < 0 ? kf + N : kf;
    return true;
}

// Index of the cell nearest (x, y) in the grid, -1 off the map or for a
// non-finite coordinate (the cell test of the occupancy pre-check).
__device__ __forceinline__ int64_t map_cell(int W, int H, float x, float y)
{
    const float fx = floorf(__fadd_rn(x, 0.5f));
    const float fy = floorf(__fadd_rn(y, 0.5f));
    if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) return -1;
    return (int64_t)(int)fy * W + (int)fx;
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

// Keys per 32-byte node (K = 2^LK) and root fan-out R held in the header.
template <typename KT> struct KeyT;
template <> struct KeyT<float> {
    static constexpr int LK = 3;
    static constexpr int K = 8;
    static constexpr int R = 6;
};
template <> struct KeyT<uint16_t> {
    static constexpr int LK = 4;
    static constexpr int K = 16;
    static constexpr int R = 12;
};

// Nodes at level l of a bin with L0 leaves (level 0 = leaves).
__host__ __device__ __forceinline__ uint32_t level_count(uint32_t L0, int LK, int l)
{
    return (uint32_t)(((uint64_t)(L0 - 1) >> (LK * l)) + 1);
}

// Internal levels stored in the run: the smallest h whose level fits under
// the root (at most R nodes).
__host__ __device__ __forceinline__ int run_levels(uint32_t L0, int LK, int R)
{
    int h = 0;
    while (level_count(L0, LK, h) > (uint32_t)R) ++h;
    return h;
}

__host__ __device__ __forceinline__ uint32_t internal_nodes(uint32_t n, int LK, int R)
{
    if (n == 0) return 0;
    uint32_t L0 = ((n - 1) >> LK) + 1;
    int h = run_levels(L0, LK, R);
    uint32_t t = 0;
    for (int l = 1; l <= h; ++l) t += level_count(L0, LK, l);
    return t;
}

__host__ __device__ __forceinline__ uint32_t bin_nodes(uint32_t n, int LK, int R)
{
    if (n == 0) return 0;
    return internal_nodes(n, LK, R) + ((n - 1) >> LK) + 1;
}

// Loads of a 32-byte node: one 256-bit load (CDDT_LD_V8) or two 128-bit
// loads; `pol` is an L2 cache policy applied when CDDT_LD_HINT is set.
#ifndef CDDT_LD_V8
#define CDDT_LD_V8 1
#endif
#ifndef CDDT_LD_HINT
#define CDDT_LD_HINT 1
#endif
__device__ __forceinline__ void ld_node(const void *p, uint32_t (&w)[8])
{
#if CDDT_LD_V8
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(p));
#else
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
#endif
}
__device__ __forceinline__ void ld_node(const void *p, uint64_t pol, uint32_t (&w)[8])
{
#if CDDT_LD_HINT && CDDT_LD_V8
    asm("ld.global.nc.L2::cache_hint.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(p), "l"(pol));
#elif CDDT_LD_HINT
    asm("ld.global.nc.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p), "l"(pol));
    asm("ld.global.nc.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(reinterpret_cast<const char *>(p) + 16), "l"(pol));
#else
    (void)pol;
    ld_node(p, w);
#endif
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol = 0;
#if CDDT_LD_HINT
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#endif
    return pol;
}

// The default L2 priority, for casts whose gathers move through the store
// one slice at a time (nothing should outlive its slice in L2).
__device__ __forceinline__ uint64_t policy_evict_normal()
{
    uint64_t pol = 0;
#if CDDT_LD_HINT
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
#endif
    return pol;
}

// Leaves are read with the evict-first priority: under a stream of leaf
// reads that misses L2 (uniformly spread queries) they are the first lines
// to go, ahead of the bin headers and internal nodes.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol = 0;
#if CDDT_LD_HINT
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#endif
    return pol;
}

// Key i of a bin from its leaf run (scalar load).
template <typename KT>
__device__ __forceinline__ float bin_key(const MapView &m, uint32_t off, uint32_t n, int i, float X)
{
    constexpr int LK = KeyT<KT>::LK;
    const size_t leaf = (size_t)off + internal_nodes(n, LK, KeyT<KT>::R);
    if (sizeof(KT) == 4) return __ldg(chk_store(m, reinterpret_cast<const float *>(m.store) + (leaf << 3) + i, 4));
    return dequantise(__ldg(chk_store(m, reinterpret_cast<const uint16_t *>(m.store) + (leaf << 4) + i, 2)), X,
                      m.invQ);
}

// Search result: index of the first key > x (Upper) or >= x (!Upper) in the
// bin, n when none; the key at that index (when < n) and the key just before
// it (when the index is > 0), which the paired reverse beam uses.
struct SearchResult {
    int idx;
    float at;    // key[idx]
    float prev;  // key[idx - 1]
};

// Comparison of node keys against a query abscissa.  float32 keys compare
// directly; 16-bit keys compare as integers against the exact threshold:
// value(key) = key / Q - X is exact in float32, so value(key) <= x iff
// key <= floor((x + X) Q) and value(key) < x iff key <= ceil((x + X) Q) - 1.
// X is an integer and Q a power of two, so X Q is an integer and the
// threshold is floor(x Q) + X Q (ceil(x Q) + X Q - 1), every step exact in
// float32 (x + X itself would round).
template <typename KT, bool Upper> struct Cmp;
template <bool Upper> struct Cmp<float, Upper> {
    float x;
    __device__ __forceinline__ Cmp(const MapView &, float x_, float) : x(x_) {}
    __device__ __forceinline__ bool le(uint32_t bits) const
    {
        float v = __uint_as_float(bits);
        return Upper ? (v <= x) : (v < x);
    }
};
template <bool Upper> struct Cmp<uint16_t, Upper> {
    int t;
    __device__ __forceinline__ Cmp(const MapView &m, float x, float X)
    {
        // floor((x + X) Q) = floor(x Q) + X Q because X Q is an integer; x Q
        // is exact (Q a power of two >= 1) and, for a cast from inside the
        // map, both sums are integers below 2^24 in magnitude, so exact too
        const float f = __fmul_rn(x, m.Q), xq = __fmul_rn(X, m.Q);
        const float tt = Upper ? __fadd_rn(floorf(f), xq) : __fsub_rn(__fadd_rn(ceilf(f), xq), 1.0f);
        t = (int)fminf(fmaxf(tt, -1.0f), 65536.0f);
    }
    __device__ __forceinline__ bool le(uint32_t key) const { return (int)key <= t; }
};

template <typename KT>
__device__ __forceinline__ float key_value(const MapView &m, uint32_t raw, float X)
{
    if (sizeof(KT) == 4) return __uint_as_float(raw);
    return dequantise(raw, X, m.invQ);
}

// Keys of a node in ascending order as raw 32-bit words (float bits or
// zero-extended uint16), NK = R for a header, K for a node.
template <typename KT, int NK>
__device__ __forceinline__ void unpack(const uint32_t *w, uint32_t (&k)[NK])
{
    if (sizeof(KT) == 4) {
#pragma unroll
        for (int i = 0; i < NK; ++i) k[i] = w[i];
    } else {
#pragma unroll
        for (int i = 0; i < NK / 2; ++i) {
            k[2 * i] = w[i] & 0xffffu;
            k[2 * i + 1] = w[i] >> 16;
        }
    }
}

// Number of a node's keys below the query when it is known to be at most 7
// (float32 keys, ascending): three comparisons, each choosing the key the
// next one looks at.  Below the root the chosen child's largest key is not
// below the query, so one of its keys never is.
template <bool Upper>
__device__ __forceinline__ int count_below7(const uint32_t (&w)[8], const Cmp<float, Upper> &cmp)
{
    const bool b2 = cmp.le(w[3]);
    const bool b1 = cmp.le(b2 ? w[5] : w[1]);
    const uint32_t lo = b1 ? w[2] : w[0], hi = b1 ? w[6] : w[4];
    const bool b0 = cmp.le(b2 ? hi : lo);
    return (b2 ? 4 : 0) + (b1 ? 2 : 0) + (b0 ? 1 : 0);
}

// The same count for a float32 leaf, with the keys either side of the
// answer taken from the registers: at = key[c] and prev = key[c - 1].  The
// third comparison looked at key[c] or key[c - 1]; the other one is an odd
// key chosen by the first two comparisons.  prev_here is false for c = 0
// (prev then sits at the end of the previous leaf).
template <bool Upper>
__device__ __forceinline__ int leaf_count7(const uint32_t (&w)[8], const Cmp<float, Upper> &cmp, uint32_t &at,
                                           uint32_t &prev, bool &prev_here)
{
    const bool b2 = cmp.le(w[3]);
    const uint32_t m2 = b2 ? w[5] : w[1];           // key[4 b2 + 1]
    const bool b1 = cmp.le(m2);
    const uint32_t lo = b1 ? w[2] : w[0], hi = b1 ? w[6] : w[4];
    const uint32_t m3 = b2 ? hi : lo;                // key[4 b2 + 2 b1]
    const bool b0 = cmp.le(m3);
    const uint32_t up = b1 ? (b2 ? w[7] : w[3]) : m2;  // key[4 b2 + 2 b1 + 1]
    const uint32_t dn = b1 ? m2 : w[3];              // key[4 b2 + 2 b1 - 1] (b2 set when !b1)
    at = b0 ? up : m3;
    prev = b0 ? m3 : dn;
    prev_here = b0 || b1 || b2;
    return (b2 ? 4 : 0) + (b1 ? 2 : 0) + (b0 ? 1 : 0);
}

// Number of the six header keys w[2..7] below the query (0..6), the same way:
// a count of 6 (every key below) needs no third comparison.
template <bool Upper>
__device__ __forceinline__ int count_below6(const uint32_t (&w)[8], const Cmp<float, Upper> &cmp)
{
    const bool b2 = cmp.le(w[5]);
    const bool b1 = cmp.le(b2 ? w[7] : w[3]);
    const uint32_t lo = b1 ? w[4] : w[2];
    const bool b0 = !(b2 && b1) && cmp.le(b2 ? w[6] : lo);
    return (b2 ? 4 : 0) + (b1 ? 2 : 0) + (b0 ? 1 : 0);
}

// 16-bit keys: key j of a node is half (j & 1) of word j >> 1; a header's
// key i sits where node key i + 4 would.  Word and key selection by a select
// tree (a register array indexed at run time would go to local memory).
__device__ __forceinline__ uint32_t sel_word(const uint32_t (&w)[8], int i)
{
    const bool o = i & 1;
    const uint32_t a = o ? w[1] : w[0], b = o ? w[3] : w[2], c = o ? w[5] : w[4], d = o ? w[7] : w[6];
    const uint32_t e = (i & 2) ? b : a, f = (i & 2) ? d : c;
    return (i & 4) ? f : e;
}
__device__ __forceinline__ uint32_t key16_at(const uint32_t (&w)[8], int j)
{
    return (sel_word(w, j >> 1) >> ((j & 1) * 16)) & 0xffffu;
}

// Number of a 16-bit node's keys below the query when it is at most 15 (a
// node below the root: its largest key is its separator, not below the
// query): four comparisons, each choosing the key the next one looks at.
template <bool Upper>
__device__ __forceinline__ int count_below15(const uint32_t (&w)[8], const Cmp<uint16_t, Upper> &cmp)
{
    const bool b3 = cmp.le(w[3] >> 16);                    // key 7
    const bool b2 = cmp.le((b3 ? w[5] : w[1]) >> 16);      // key 8 b3 + 3
    const uint32_t lo = b2 ? w[2] : w[0], hi = b2 ? w[6] : w[4];
    const bool b1 = cmp.le((b3 ? hi : lo) >> 16);          // key 8 b3 + 4 b2 + 1
    const int wi = (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
    const bool b0 = cmp.le(sel_word(w, wi) & 0xffffu);     // key 2 wi
    return 2 * wi + (b0 ? 1 : 0);
}

// The same count for a 16-bit leaf, with the keys either side of the answer
// taken from what the search already holds: at = key[c], prev = key[c - 1]
// (the last comparison read key 2 wi, and key 2 wi - 1 is the key of the
// latest comparison that went the other way); prev_here is false for c = 0.
template <bool Upper>
__device__ __forceinline__ int leaf_count15(const uint32_t (&w)[8], const Cmp<uint16_t, Upper> &cmp, uint32_t &at,
                                            uint32_t &prev, bool &prev_here)
{
    const uint32_t k7 = w[3] >> 16;
    const bool b3 = cmp.le(k7);
    const uint32_t k3 = (b3 ? w[5] : w[1]) >> 16;          // key 8 b3 + 3
    const bool b2 = cmp.le(k3);
    const uint32_t lo = b2 ? w[2] : w[0], hi = b2 ? w[6] : w[4];
    const uint32_t k1 = (b3 ? hi : lo) >> 16;              // key 8 b3 + 4 b2 + 1
    const bool b1 = cmp.le(k1);
    const int wi = (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
    const uint32_t word = sel_word(w, wi);
    const uint32_t k0 = word & 0xffffu;                    // key 2 wi
    const bool b0 = cmp.le(k0);
    at = b0 ? word >> 16 : k0;
    prev = b0 ? k0 : (b1 ? k1 : (b2 ? k3 : k7));
    prev_here = b0 || b1 || b2 || b3;
    return 2 * wi + (b0 ? 1 : 0);
}

// The same for the 12 keys of a 16-bit header (0..12 below), positions
// 12..15 counting as above every query.
template <bool Upper>
__device__ __forceinline__ int count_below12(const uint32_t (&w)[8], const Cmp<uint16_t, Upper> &cmp)
{
    const bool b3 = cmp.le(w[5] >> 16);                    // key 7
    const bool b2 = cmp.le((b3 ? w[7] : w[3]) >> 16);      // key 8 b3 + 3
    const bool top = b3 && b2;                             // keys 13 and 12 do not exist
    const bool b1 = !top && cmp.le((b3 ? w[6] : (b2 ? w[4] : w[2])) >> 16);  // key 8 b3 + 4 b2 + 1
    const int wi = (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
    const bool o = wi & 1;
    const uint32_t x0 = o ? w[3] : w[2], x1 = o ? w[5] : w[4], x2 = o ? w[7] : w[6];
    const uint32_t word = (wi & 4) ? x2 : ((wi & 2) ? x1 : x0);
    const bool b0 = !top && cmp.le(word & 0xffffu);        // key 8 b3 + 4 b2 + 2 b1
    return 2 * wi + (b0 ? 1 : 0);
}

// Number of a node's keys below the query (keys ascending, padding above).
template <typename KT, bool Upper>
__device__ __forceinline__ int count_below(const uint32_t (&w)[8], int from, const Cmp<KT, Upper> &cmp)
{
    int c = 0;
    if (sizeof(KT) == 4) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i >= from) c += cmp.le(w[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i >= from) c += cmp.le(w[i] & 0xffffu) + cmp.le(w[i] >> 16);
    }
    return c;
}

// Key at element index e of an array of KT (scalar load, usually an L1 hit).
template <typename KT, bool InHdr = false>
__device__ __forceinline__ float load_key(const MapView &m, const void *base, int64_t e, float X)
{
    if (sizeof(KT) == 4) {
        const float *p = reinterpret_cast<const float *>(base) + e;
        return __ldg(InHdr ? chk_hdr(m, p, 4) : chk_store(m, p, 4));
    }
    const uint16_t *p = reinterpret_cast<const uint16_t *>(base) + e;
    return dequantise(__ldg(InHdr ? chk_hdr(m, p, 2) : chk_store(m, p, 2)), X, m.invQ);
}

// Search one bin through its header and tree (layout above): count the keys
// below the query at each level, then load the answer's neighbours from the
// leaf (the leaves are contiguous, so key idx - 1 sits just before key idx).
// kb receives the bin's size.
template <typename KT, bool Upper>
__device__ __forceinline__ SearchResult tree_search(const MapView &m, uint32_t g, float x, float X, uint64_t pol,
                                                    int &kb)
{
    constexpr int LK = KeyT<KT>::LK;
    constexpr int K = KeyT<KT>::K;
    constexpr int R = KeyT<KT>::R;
    SearchResult r;
    r.idx = 0;
    r.at = kInf;
    r.prev = -kInf;
    uint32_t w[8];
    ld_node(chk_hdr(m, m.hdr + g, 32), pol, w);
    const uint32_t off = w[0], n = bin_count(w[1]);
    kb = (int)n;
    if (n == 0) return r;
    const Cmp<KT, Upper> cmp(m, x, X);
    int c;
    if constexpr (sizeof(KT) == 4) c = count_below6<Upper>(w, cmp);
    else c = count_below12<Upper>(w, cmp);
    if (n <= (uint32_t)R) {  // the keys themselves are in the header
        // padding never compares below an in-map query; the clamp keeps the
        // answer inside the bin regardless
        r.idx = min(c, (int)n);
        if constexpr (sizeof(KT) == 4) {
            const void *keys = reinterpret_cast<const uint32_t *>(m.hdr + g) + 2;
            if (r.idx < (int)n) r.at = load_key<KT, true>(m, keys, r.idx, X);
            if (r.idx > 0) r.prev = load_key<KT, true>(m, keys, r.idx - 1, X);
        } else {  // from the header's registers
            if (r.idx < (int)n) r.at = dequantise(key16_at(w, r.idx + 4), X, m.invQ);
            if (r.idx > 0) r.prev = dequantise(key16_at(w, r.idx + 3), X, m.invQ);
        }
        return r;
    }
    const uint32_t L0 = ((n - 1) >> LK) + 1;
    const int h = (int)((w[1] >> 24) & 15u);     // stored levels, from the header
    const int cnt_h = (int)(w[1] >> 28);         // the root's children
    const char *run = reinterpret_cast<const char *>(m.store) + ((size_t)off << 5);
    if (c >= cnt_h) {  // every key is below the query
        r.idx = (int)n;
        r.prev = load_key<KT>(m, run + ((size_t)internal_nodes(n, LK, R) << 5), (int64_t)n - 1, X);
        return r;
    }
    uint32_t loff = 0, k = (uint32_t)c;
    uint32_t cnt = (uint32_t)cnt_h;  // nodes at the current level
    for (int l = h; l >= 1; --l) {
        ld_node(chk_store(m, run + ((size_t)(loff + k) << 5), 32), pol, w);
        int cc;
        if constexpr (sizeof(KT) == 4) cc = count_below7<Upper>(w, cmp);
        else cc = count_below15<Upper>(w, cmp);
        loff += cnt;
        cnt = ((L0 - 1) >> (LK * (l - 1))) + 1;  // nodes one level down
        k = k * K + (uint32_t)cc;
        // float32 padding never compares below a query; 16-bit padding could
        // only for a query beyond the map, and the clamp keeps that inside
        if (sizeof(KT) != 4) k = min(k, cnt - 1);
    }
    // leaf (loff is now the number of internal nodes)
    const char *leaf = run + ((size_t)(loff + k) << 5);
    ld_node(chk_store(m, leaf, 32), policy_evict_first(), w);
    if constexpr (sizeof(KT) == 4) {
        uint32_t at, prev;
        bool prev_here;
        c = leaf_count7<Upper>(w, cmp, at, prev, prev_here);
        r.idx = (int)(k * K) + c;  // <= n: padding never compares below a query
        if (r.idx < (int)n) r.at = __uint_as_float(at);
        if (prev_here) r.prev = __uint_as_float(prev);
        else if (k > 0) r.prev = load_key<KT>(m, leaf, -1, X);
    } else {
        // at most 15 keys of the chosen leaf are below (its largest is its
        // separator); the answer's neighbours come from the registers
        uint32_t at, prev;
        bool prev_here;
        c = leaf_count15<Upper>(w, cmp, at, prev, prev_here);
        const int raw = (int)(k * K) + c;
        r.idx = min(raw, (int)n);  // padding is below only a query beyond the map
        if (r.idx < (int)n) r.at = dequantise(at, X, m.invQ);
        if (raw > (int)n) r.prev = load_key<KT>(m, leaf, (int64_t)n - 1 - (int64_t)(k * K), X);
        else if (prev_here) r.prev = dequantise(prev, X, m.invQ);
        else if (k > 0) r.prev = load_key<KT>(m, leaf, -1, X);
    }
    return r;
}

// Branch-free binary search of the bin's sorted leaf run (same answers).
template <typename KT, bool Upper>
__device__ __forceinline__ SearchResult binary_search(const MapView &m, uint32_t g, float x, float X, int &kb)
{
    SearchResult r;
    r.idx = 0;
    r.at = kInf;
    r.prev = -kInf;
    const uint2 on = __ldg(chk_hdr(m, reinterpret_cast<const uint2 *>(m.hdr + g), 8));
    const uint32_t off = on.x;
    const int n = (int)bin_count(on.y);
    kb = n;
    if (n == 0) return r;
    int base = 0, len = n;
    while (len > 1) {
        int half = len >> 1;
        float v = bin_key<KT>(m, off, n, base + half - 1, X);
        base = (Upper ? (v <= x) : (v < x)) ? base + half : base;
        len -= half;
    }
    float v = bin_key<KT>(m, off, n, base, X);
    int idx = base + (Upper ? (v <= x) : (v < x));
    r.idx = idx;
    if (idx < n) r.at = (idx == base) ? v : bin_key<KT>(m, off, n, idx, X);
    if (idx > 0) r.prev = (idx - 1 == base) ? v : bin_key<KT>(m, off, n, idx - 1, X);
    return r;
}

// The search layout is a template parameter (SEARCH = CDDT_SEARCH_*), so a
// kernel carries the code of one layout only.
template <typename KT, bool Upper, int SEARCH>
__device__ __forceinline__ SearchResult bin_search(const MapView &m, uint32_t g, float x, float X, uint64_t pol,
                                                   int &kb)
{
    if (SEARCH == CDDT_SEARCH_BINARY) return binary_search<KT, Upper>(m, g, x, X, kb);
    return tree_search<KT, Upper>(m, g, x, X, pol, kb);
}

// ------------------------------------------------------------ one ray cast

// Result of casting one beam: range and its derivative direction.
struct Cast {
    float r;         // clamped range
    float dzx, dzy;  // d r / d(x, y): -(c, s) forward, +(c, s) backward, 0 if clamped / miss
    int kb;          // bin size searched (-1: none)
};

// Cast from an in-map free cell position (pre-check already passed) in
// direction k.  One search; if `pair` is set, the opposite direction k + N/2
// is answered from the same search (Section IV-C: index i - 1).
template <typename KT, int SEARCH>
__device__ __forceinline__ void cast_pair(const MapView &m, float x, float y, int k, bool pair, uint64_t pol,
                                          Cast &fwd_out, Cast &bwd_out, bool &k_is_fwd)
{
    const int S = m.S;
    const bool bwd = k >= S;
    const int s = bwd ? k - S : k;
    k_is_fwd = !bwd;
    // float32 keys read the slice record's first 16 bytes; 16-bit keys the
    // whole 32 (the key offset X with it, one load)
    float4 sa;
    float X = 0.0f;
    if constexpr (sizeof(KT) == 4) {
        sa = __ldg(chk_slice(m, reinterpret_cast<const float4 *>(m.slices + s), 16));
    } else {
        uint32_t w[8];
        ld_node(chk_slice(m, m.slices + s, 32), w);
        sa = make_float4(__uint_as_float(w[0]), __uint_as_float(w[1]), __uint_as_float(w[2]), __uint_as_float(w[3]));
        X = __uint_as_float(w[4]);
    }
    const float c = sa.x, sn = sa.y;
    const uint32_t Tnb = __float_as_uint(sa.w);
    const int T = (int)(Tnb & 0xffffu), nb = (int)(Tnb >> 16);
    float xr, yr;
    project(x, y, c, sn, xr, yr);
    const int b = query_bin(yr, T);
    Cast f, r;
    f.r = r.r = m.max_range;
    f.dzx = f.dzy = r.dzx = r.dzy = 0.0f;
    f.kb = r.kb = -1;
    if (b >= 0 && b < nb) {
        const uint32_t g = __float_as_uint(sa.z) + (uint32_t)b;
        int kb;
        if (!bwd || pair) {
            // forward: first key > x' (upper bound)
            SearchResult sr = bin_search<KT, true, SEARCH>(m, g, xr, X, pol, kb);
            if (sr.idx < kb) {
                float d = __fsub_rn(sr.at, xr);
                if (d < m.max_range) { f.r = d; f.dzx = -c; f.dzy = -sn; }
            }
            if (pair) {
                // backward from the same search: last key < x'
                float pv = sr.prev;
                int j = sr.idx - 1;
                if (j >= 0 && pv == xr) {
                    const uint2 on = __ldg(chk_hdr(m, reinterpret_cast<const uint2 *>(m.hdr + g), 8));
                    while (j >= 0 && pv == xr) {
                        --j;
                        if (j >= 0) pv = bin_key<KT>(m, on.x, bin_count(on.y), j, X);
                    }
                }
                if (j >= 0) {
                    float d = __fsub_rn(xr, pv);
                    if (d < m.max_range) { r.r = d; r.dzx = c; r.dzy = sn; }
                }
            }
        } else {
            // backward only: last key < x' = (first key >= x') - 1
            SearchResult sr = bin_search<KT, false, SEARCH>(m, g, xr, X, pol, kb);
            if (sr.idx > 0) {
                float d = __fsub_rn(xr, sr.prev);
                if (d < m.max_range) { r.r = d; r.dzx = c; r.dzy = sn; }
            }
        }
        f.kb = r.kb = kb;
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
    float hit_a;   // z_hit / (sigma sqrt(2 pi)): the weighted hit peak
    float hit_k2;  // log2(e) / (2 sigma^2): hit exponent in base 2
    float lam_l2;  // lambda log2(e)
    float pad;
};

inline BeamConsts make_beam_consts(const cddt_beam_model &m)
{
    const double LOG2E = 1.4426950408889634;
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
    b.hit_a = (float)((double)m.z_hit / (sig * 2.5066282746310002));
    b.hit_k2 = (float)(LOG2E / (2.0 * sig * sig));
    b.lam_l2 = (float)((double)m.lambda_short * LOG2E);
    b.pad = 0.0f;
    return b;
}

// Per-beam terms that depend on the measurement only; staged in shared
// memory as one float4 per beam together with the beam's angle offset.
struct BeamObs {
    float z;      // measured range clamped to [0, max_range]
    float s_lz;   // z_short lambda e^{-lambda z}
    float c_mr;   // z_max [z >= max] + z_rand [z < max] / max_range
};

__device__ __forceinline__ BeamObs beam_obs(const BeamConsts &m, float obs)
{
    BeamObs o;
    float z = fminf(fmaxf(obs, 0.0f), m.max_range);
    o.z = z;
    o.s_lz = m.z_short * (m.lam * expf(-m.lam * z));
    o.c_mr = (z >= m.max_range) ? m.z_max : m.z_rand * m.inv_max_range;
    return o;
}

// The hardware base-2 exponential, logarithm and reciprocal (PTX ex2, lg2,
// rcp .approx): relative errors of a few 2^-23, results below 2^-126 flushed.
__device__ __forceinline__ float hw_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_log2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1 - e^{-u} for u >= 0 given e = e^{-u}.  Below u = 1/2 the difference
// would cancel, so it is the Maclaurin series u - u^2/2! + u^3/3! - ...
// through u^9 (truncation below 1.1e-8 relative there); above, 1 - e loses
// nothing (e <= 0.61).
__device__ __forceinline__ float one_minus_exp_neg(float u, float e)
{
    float t = 2.7557319e-6f;                 //  1/9!
    t = fmaf(t, -u, 2.4801587e-5f);          //  1/8!
    t = fmaf(t, -u, 1.9841270e-4f);          //  1/7!
    t = fmaf(t, -u, 1.3888889e-3f);          //  1/6!
    t = fmaf(t, -u, 8.3333333e-3f);          //  1/5!
    t = fmaf(t, -u, 4.1666667e-2f);          //  1/4!
    t = fmaf(t, -u, 1.6666667e-1f);          //  1/3!
    t = fmaf(t, -u, 0.5f);                   //  1/2!
    t = fmaf(t, -u, 1.0f);
    return u < 0.5f ? u * t : 1.0f - e;
}

constexpr float kLn2 = 0.69314718055994531f;

// log2 p(z | z*) and, when wanted, d ln p / d z* (Section VI's beam model:
// a Gaussian hit, an exponential short reading normalised on [0, z*], a
// max-range spike and a uniform floor).  Callers multiply the summed log2
// by ln 2 once per particle.  The exponentials, the reciprocal and the
// logarithm use the hardware approximations: their error, a few 1e-7 of
// ln p per beam, is far below the 1e-5 relative parity bar on the
// particle's sum.  Every term is evaluated and selected, without branches.
template <bool Grad>
__device__ __forceinline__ float beam_log2p(const BeamConsts &m, const BeamObs &o, float zs, float &dlogp)
{
    const float d = o.z - zs;
    float ph = m.hit_a * hw_exp2(-(d * d) * m.hit_k2);  // z_hit p_hit
    float dhit = 0.0f;
    if (m.trunc) {
        float a = (m.max_range - zs) * m.inv_sig;
        float b = -zs * m.inv_sig;
        float D = normcdff(a) - normcdff(b);
        ph = ph / D;
        if (Grad) {
            const float r2pi = 0.3989422804014327f;
            float dD = (r2pi * expf(-0.5f * b * b) - r2pi * expf(-0.5f * a * a)) * m.inv_sig;
            dhit = ph * (d * m.inv_s2 - dD / D);
        }
    } else if (Grad) {
        dhit = ph * d * m.inv_s2;
    }
    // z_short p_short = z_short lambda e^{-lambda z} / (1 - e^{-lambda z*}), 0 < z <= z*
    const float e = hw_exp2(-zs * m.lam_l2);
    const float inv = hw_rcp(one_minus_exp_neg(m.lam * zs, e));
    const bool short_on = zs > 0.0f && o.z <= zs;
    const float ps = short_on ? o.s_lz * inv : 0.0f;
    const float p = ph + ps + o.c_mr;
    if (Grad) {
        const float dshort = (zs > 0.0f && o.z < zs) ? -m.lam * o.s_lz * e * inv * inv : 0.0f;
        dlogp = (dhit + dshort) / p;
    }
    return hw_log2(p);
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
    uint64_t generation = 0;  // bumped whenever the store, its layout or the search changes
    int64_t total_bins = 0;
    int64_t n_zp = 0;          // zero points (host copy, exact after each sync point)
    int64_t n_edge = 0;
    int64_t store_nodes = 0;   // nodes in use
    int64_t store_cap = 0;     // nodes allocated
    int64_t max_bin = 0;
    float build_ms = 0, prune_ms = 0, update_ms = 0;
    // device buffers owned by the handle
    cddt::SliceInfo *slices = nullptr;
    cddt::BinHdr *hdr = nullptr;
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
    // kept by updates: the previous store (reused as the next update's
    // target) and grow-only workspaces
    void *spare = nullptr;
    int64_t spare_nodes = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *ws_keys = nullptr;
    size_t ws_keys_bytes = 0;

    cddt::MapView view() const
    {
        cddt::MapView v;
        v.slices = slices;
        v.hdr = hdr;
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
#if CDDT_CHECKED
        v.hdr_bytes = (int64_t)sizeof(cddt::BinHdr) * total_bins;
        // CDDT_FAULT=bounds: report half the store in use, so that the checks
        // fire on valid reads (the reads themselves stay inside the buffer)
        const char *f = std::getenv("CDDT_FAULT");
        v.store_bytes = 32 * ((f && !std::strcmp(f, "bounds")) ? store_nodes / 2 : store_cap);
        v.status = status;
#endif
        return v;
    }
};

// Host helpers shared by the translation units.
namespace cddt {
cddt_status cuda_status(cudaError_t e);
// Streaming multiprocessors of the current device, queried once per device
// and cached (cddt_build.cu).  Grid caps are multiples of it; when the query
// fails it returns 1, which only narrows a grid-stride launch.
int sm_count();
// Build the sorted, tree-indexed store from per-bin key lists; implemented in
// cddt_build.cu and reused by prune and update.
cddt_status build_index(cddt_s *h, cudaStream_t st);
}  // namespace cddt

#define CDDT_CUDA(call)                                                       \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return cddt::cuda_status(e_);                  \
    } while (0)

#define CDDT_TRY(call)                                                        \
    do {                                                                      \
        cddt_status r_ = (call);                                              \
        if (r_ != CDDT_OK) return r_;                                         \
    } while (0)
