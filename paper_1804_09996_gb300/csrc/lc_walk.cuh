// Device-side definitions of the search walk (shared by the element-type translation units
// lc_walk_f32.cu / lc_walk_f16.cu and by lc_search.cu): kernel arguments, shared-memory
// layouts, the scoring helpers and the walk kernel template, and the host templates that
// configure and launch one instantiation.  Not part of the ABI.
//
// walk_kernel (one warp per query; persistent CTAs take queries from an atomic counter)
//   - y' = R y from the rotation kernel (or rotated here, for the walk without allocation);
//   - the walk distance is the ADC distance ||y' - c1(x)||^2 of Section 4.1: the sum over
//     level-1 sub-spaces j of ||y'^j - C1_j[c_j]||^2, each term computed in FP32 from the
//     codebook C1, which every CTA keeps once in shared memory (a per-query table of the same
//     terms would cost 32-64 KB of shared memory per query in flight); with FQ the distance is
//     to the full two-level decode c1 + c2;
//   - greedy descent of the upper HNSW levels, then best-first search of level 0 with result
//     set W of size ef' (Section 2), in one loop with a single scoring call site.  W is a
//     sorted list of (distance, id) keys with an "expanded" flag: each step expands the best
//     unexpanded member (or the `beam` best) of W, scores all their unvisited neighbours at
//     once (one per lane) and merges them into W keeping the ef' best.  With one expansion
//     per step this expands exactly the nodes, in exactly the order, of the two-set
//     formulation (candidate heap C + result heap W);
//   - exact visited set: open-addressing hash in shared memory, spilling to a per-warp table
//     in global memory when it fills;
//   - writes the shortlist (the R best of W, Section 4.1 two-stage search) or, without
//     refinement, the top-k directly;
//   - ordered search: a first launch (mode 1) runs only the upper-level descent of every query
//     and records where it enters level 0; a second (mode 2) runs the level-0 searches from
//     those entry nodes in the order the host sorted them (the queries whose entry node is
//     farthest from them first: they tend to walk longest, so the launch no longer ends with a
//     few long walks on an otherwise idle GPU).  Each query's result is the same as in one
//     launch (mode 0): the entry node and its distance are the ones the descent computes.
//
// FP32 walk distance: lane l holds the term of sub-space l (M1 = 32), of l mod 16 (M1 = 16)
// or the sum of sub-spaces l and l + 32 (M1 = 64), each term summed over its coordinates in
// order; the 32 lane values are added pairwise, lanes differing in bit 3 first, then bits 2,
// 1, 0 and 4.  The order is the same for every node, so a node's distance does not depend on
// where or with how many others it is scored.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lc_device.h"

namespace lc {

#define FULL 0xffffffffu

// ------------------------------------------------------------------------------------------
// Kernel arguments
struct SplitTab {
    uint16_t off[64];
    uint8_t len[64];
};

struct WalkArgs {
    const float *Q;
    const uint8_t *Q8;     // non-null: the queries are uint8 [nq][d] (Q unused)
    const int32_t *efq;    // non-null: per-query efSearch [nq], clamped to 1..efp
    int k;
    int64_t nq;
    int d;
    const float *Rt, *C1;
    const __half *C1h;     // the same codebook in FP16 (FP16 mode); both in the walk's layout
    const uint8_t *codes1;
    const int32_t *adj0, *upper_off, *upper_adj;
    int32_t ep;
    int max_level;
    int efp;          // ef' = max(ef, k); with efq, the largest any query may use
    int efcap;        // efp rounded up to a multiple of 32
    int R;            // shortlist length (refine) or k (no refinement)
    int refine;
    int beam;         // expansions per step (1: the plain walk)
    int tcap;         // > 0: stop once that many level-0 distances were computed
    int hash_log;     // shared-memory visited table: 2^hash_log entries
    int spill_log;    // global spill table per warp: 2^spill_log entries
    int32_t *spill;
    const float *yq_in;    // non-null: y' = R y computed by rotate_kernel (read, not recomputed)
    float *yq_out;
    int32_t *short_out;
    int32_t *ids_out;
    float *dists_out;
    int32_t *stats_out;
    int32_t *status;
    unsigned long long *counter;   // next query to take (reset to 0 before each launch)
    SplitTab s1;
    // walk on the full two-level decode (kernels instantiated with FQ = true)
    const float *C2;       // [256][d] FP32, read through the cache
    const __half *C2h;     // [256][d] FP16, copied into shared memory
    const uint8_t *codes2b;
    int M2P;
    uint8_t sub2[256];     // level-2 sub-space of each coordinate
    // ordered search (see walk_kernel): 0 = the whole walk; 1 = the upper levels only, writing
    // each query's level-0 entry node, its walk distance and the upper-level evaluations to
    // seed / seed_d / seed_up; 2 = level 0 only, from those, queue position i taking query
    // order[i] (order may be null: position i is query i)
    int mode;
    const int32_t *order;
    const __half *tab;     // table form: the queries' ADC tables [nq][256][M1] (FP16)
    int32_t *seed, *seed_up;
    float *seed_d;
};

constexpr int MAX_WALK_WARPS = 16;       // warps (queries in flight) per CTA

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared memory of the walk kernel: the level-1 codebook C1 [256][d] once per CTA, then one
// region per warp.
struct WalkSmem {
    size_t yq, stage, wkey, wflag, cand, cunsorted, slot, rowbuf, hash, total;
};

// Layout of the walk's level-1 codebook in shared memory, chosen so that a lane's sub-space
// term takes few loads and the lanes of one shared-memory phase hit distinct banks:
//  0 (row-major): row c holds centroid c of every sub-space in its own coordinates ([256][d]).
//    Used in FP32 with 3 or 6 dimensions per sub-space (3 j + u mod 32 permutes the lanes)
//    and for non-uniform splits.
//  1 (interleaved): the P values (D1 rounded up to 2 or 8) of centroid c in sub-space j sit
//    at (c * M1 + j) * P: one vector load.  FP32 and FP16 with 2 dimensions, FP16 with 6.
//  2 (split, FP16 with 3 dimensions): the first two values as a half2 array [256][M1], the
//    third as a half array [256][M1] behind it: two loads, no padding.
__host__ __device__ constexpr int walk_layout(int D1, int es)
{
    return D1 == 0 ? 0 : D1 == 2 ? 1 : es == 4 ? 0 : D1 == 3 ? 2 : 1;
}
__host__ __device__ constexpr int walk_pad(int D1) { return D1 <= 2 ? 2 : (D1 <= 4 ? 4 : 8); }
// bytes of the level-1 codebook in shared memory (es = 4: FP32, es = 2: FP16)
__host__ __device__ inline size_t walk_c1_bytes(int d, int M1, int D1, size_t es)
{
    const int L = walk_layout(D1, (int)es);
    const size_t n = L == 1 ? (size_t)256 * M1 * walk_pad(D1) : (size_t)256 * d;
    return align_up(n * es, 128);
}
// shared memory before the per-warp regions: the walk's level-1 codebook and, for the full
// walk in FP16, C2 [256][d] behind it
__host__ __device__ inline size_t walk_cb_bytes(int d, int M1, int D1, size_t es, bool fq)
{
    return walk_c1_bytes(d, M1, D1, es) + (fq && es == 2 ? align_up((size_t)256 * d * 2, 128) : 0);
}
// compile-time sub-space width of the uniform splits 96/16, 96/32 and 128/64 (0: other)
__host__ __device__ constexpr int walk_variant_d1(int variant) { return variant == 1 ? 6 : variant == 2 ? 3 : variant == 3 ? 2 : 0; }
inline int walk_variant(int M1, int d)
{
    return (M1 == 16 && d == 96) ? 1 : (M1 == 32 && d == 96) ? 2 : (M1 == 64 && d == 128) ? 3 : 0;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }

// own_rot: the walk rotates the query itself (y' in shared memory); otherwise y' is read from
// the rotation kernel's output.  Areas whose lives do not overlap within a step share memory:
// the adjacency rows are read before the candidates are collected (the unsorted-candidate
// area), and the staged code rows are dead once the step's nodes are scored, before the
// candidates are sorted (the sorted-candidate area).  W is one buffer, merged in place.
__host__ __device__ inline WalkSmem walk_smem(int M1, int d, int efcap, int hash_log, int beam, bool own_rot,
                                             int m2p = 0)
{
    WalkSmem s;
    size_t o = 0;
    s.yq = o;        o += own_rot ? align_up((size_t)d * 4, 16) : 0;
    s.stage = o;                                       // level-1 rows, then (full walk) residual rows
    const size_t st_b = (size_t)32 * (M1 + m2p), cd_b = (size_t)32 * beam * 8;
    s.cand = o;      o += align_up(st_b > cd_b ? st_b : cd_b, 16);
    s.wkey = o;      o += (size_t)efcap * 8;
    s.wflag = o;     o += align_up((size_t)efcap, 16);
    s.cunsorted = o; o += (size_t)32 * beam * 8;
    s.rowbuf = s.cunsorted;
    s.slot = o;      o += (size_t)32 * beam * 4;
    s.hash = o;      o += ((size_t)1 << hash_log) * 4;
    s.total = align_up(o, 128);
    return s;
}

__device__ __forceinline__ uint64_t make_key(float dist, int32_t id)
{
    return ((uint64_t)__float_as_uint(dist) << 32) | (uint32_t)id;
}
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)(k & 0xffffffffu); }
__device__ __forceinline__ float key_dist(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m)
{
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    lo = __shfl_xor_sync(FULL, lo, m);
    hi = __shfl_xor_sync(FULL, hi, m);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v)
{
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        uint64_t o = shfl_xor64(v, m);
        v = o < v ? o : v;
    }
    return v;
}

// Lane bits in the order partial distances are combined: 3, 2, 1, 0, then 4.
__host__ __device__ constexpr int comb_bit(int k) { return k < 4 ? 3 - k : 4; }
__host__ __device__ constexpr int ilog2c(int s) { return s <= 1 ? 0 : 1 + ilog2c(s >> 1); }

// Sum over the 32 lanes of S per-slot contributions (S a power of two): reduce-scatter along
// the first log2(S) combination bits, all-reduce along the rest.  The addition tree of
// every slot is the same (lanes differing in bit 3 first, then 2, 1, 0, 4), whatever S.
template <int S>
__device__ __forceinline__ float reduce_slots(float (&v)[S], int lane)
{
    constexpr int LS = ilog2c(S);
#pragma unroll
    for (int k = 0; k < LS; k++) {
        const int bit = comb_bit(k);
        const int half = (S >> k) >> 1;
        const bool hi = (lane >> bit) & 1;
#pragma unroll
        for (int i = 0; i < half; i++) {
            float send = hi ? v[i] : v[i + half];
            float keep = hi ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 1 << bit);
        }
    }
    float r = v[0];
#pragma unroll
    for (int k = LS; k < 5; k++) r += __shfl_xor_sync(FULL, r, 1 << comb_bit(k));
    return r;
}

// Slot whose total lane `lane` holds after reduce_slots<S> (S = 2^LS).
__device__ __forceinline__ int slot_of_lane(int lane, int LS)
{
    int s = 0;
    for (int k = 0; k < LS; k++) s = (s << 1) | ((lane >> comb_bit(k)) & 1);
    return s;
}

// Per-lane geometry: the level-1 sub-space(s) a lane scores and the query's coordinates in
// them.  M1 = 16: sub-space lane & 15 (the two half-warps score different nodes);
// M1 = 32: sub-space lane; M1 = 64: sub-spaces lane and lane + 32.  D1 > 0: every sub-space
// has D1 coordinates (compile-time); D1 = 0: lengths read at run time (uneven splits).
template <int M1, int D1>
struct LaneGeo {
    static constexpr int NSUB = M1 == 64 ? 2 : 1;
    static constexpr int DMAX = D1 > 0 ? D1 : (M1 == 16 ? 16 : (M1 == 32 ? 8 : 4));   // d <= 256
    int off[NSUB], len[NSUB], j[NSUB];
    float y[NSUB][DMAX];
    int m2[NSUB][DMAX];          // full walk: level-2 sub-space of each of the lane's coordinates
};

__device__ __forceinline__ void half2_to_f(uint32_t w, float &a, float &b)
{
    const __half2 h = *reinterpret_cast<const __half2 *>(&w);
    a = __low2float(h);
    b = __high2float(h);
}

// The coordinates of centroid c in this lane's k-th sub-space, as FP32.
template <int M1, int D1, typename CT>
__device__ __forceinline__ void load_row(const CT *C1s, int d, int c, const LaneGeo<M1, D1> &g, int k,
                                         float (&x)[LaneGeo<M1, D1>::DMAX])
{
    constexpr int DMAX = LaneGeo<M1, D1>::DMAX;
    constexpr int LAYOUT = walk_layout(D1, (int)sizeof(CT));
    if constexpr (LAYOUT == 2) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(C1s + ((size_t)c * M1 + g.j[k]) * 2);
        half2_to_f(w, x[0], x[1]);
        x[2] = to_f(C1s[(size_t)256 * M1 * 2 + (size_t)c * M1 + g.j[k]]);
    } else if constexpr (LAYOUT == 1) {
        constexpr int P = walk_pad(D1);
        const CT *p = C1s + ((size_t)c * M1 + g.j[k]) * P;
        float t[P];
        if constexpr (sizeof(CT) == 4) {                   // FP32, P = 2
            const float2 f = *reinterpret_cast<const float2 *>(p);
            t[0] = f.x;
            t[1] = f.y;
        } else if constexpr (P == 2) {
            half2_to_f(*reinterpret_cast<const uint32_t *>(p), t[0], t[1]);
        } else {
            const uint4 w = *reinterpret_cast<const uint4 *>(p);
            half2_to_f(w.x, t[0], t[1]);
            half2_to_f(w.y, t[2], t[3]);
            half2_to_f(w.z, t[4], t[5]);
            half2_to_f(w.w, t[6], t[7]);
        }
#pragma unroll
        for (int u = 0; u < DMAX; u++) x[u] = t[u];
    } else {
        const CT *row = C1s + c * d + g.off[k];
#pragma unroll
        for (int u = 0; u < DMAX; u++) x[u] = (D1 > 0 || u < g.len[k]) ? to_f(row[u]) : 0.f;
    }
}

// ||y'^j - C1_j[c]||^2 in the fixed order of the sub-space's coordinates.
template <int M1, int D1, typename CT>
__device__ __forceinline__ float part_dist(const CT *C1s, int d, int c, const LaneGeo<M1, D1> &g, int k)
{
    float x[LaneGeo<M1, D1>::DMAX];
    load_row<M1, D1, CT>(C1s, d, c, g, k, x);
    float s = 0.f;
    if (D1 > 0) {
#pragma unroll
        for (int u = 0; u < LaneGeo<M1, D1>::DMAX; u++) {
            float df = g.y[k][u] - x[u];
            s = fmaf(df, df, s);
        }
    } else {
#pragma unroll
        for (int u = 0; u < LaneGeo<M1, D1>::DMAX; u++)
            if (u < g.len[k]) {
                float df = g.y[k][u] - x[u];
                s = fmaf(df, df, s);
            }
    }
    return s;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// The sub-space terms of two codes c0, c1 at once with packed FP32x2 arithmetic: each half
// performs exactly the scalar operations of part_dist (same rounding), two slots per
// instruction.
template <int M1, int D1, typename CT>
__device__ __forceinline__ void pair_dist(const CT *C1s, int d, int c0, int c1, const LaneGeo<M1, D1> &g,
                                          int k, float &s0, float &s1)
{
    float x0[LaneGeo<M1, D1>::DMAX], x1[LaneGeo<M1, D1>::DMAX];
    load_row<M1, D1, CT>(C1s, d, c0, g, k, x0);
    load_row<M1, D1, CT>(C1s, d, c1, g, k, x1);
    unsigned long long acc = 0ull;                   // (+0.f, +0.f)
#pragma unroll
    for (int u = 0; u < D1; u++) {
        const unsigned long long yy = pack2(g.y[k][u], g.y[k][u]);
        const unsigned long long cc = pack2(x0[u], x1[u]);
        unsigned long long df;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(yy), "l"(cc));
        asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(acc) : "l"(df), "l"(acc));
    }
    unpack2(acc, s0, s1);
}

// C2 value for the full walk: FP32 codebooks are read through the cache, FP16 ones from
// shared memory.
__device__ __forceinline__ float c2_at(const float *p) { return __ldg(p); }
__device__ __forceinline__ float c2_at(const __half *p) { return __half2float(*p); }

// Full walk: sum over this lane's coordinates t of (y'_t - (C1[c1][t] + C2[c2_m(t)][t]))^2,
// where row2 is the node's staged residual row and m(t) the level-2 sub-space of t.
template <int M1, int D1, typename CT>
__device__ __forceinline__ float part_full(const CT *C1s, const CT *C2, int d, int c, const uint8_t *row2,
                                           const LaneGeo<M1, D1> &g, int k)
{
    float x[LaneGeo<M1, D1>::DMAX];
    load_row<M1, D1, CT>(C1s, d, c, g, k, x);
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < LaneGeo<M1, D1>::DMAX; u++) {
        if (D1 == 0 && u >= g.len[k]) continue;
        const float v = x[u] + c2_at(C2 + (int)row2[g.m2[k][u]] * d + g.off[k] + u);
        const float df = g.y[k][u] - v;
        s = fmaf(df, df, s);
    }
    return s;
}

// Sub-space terms of S slots (S = 16 or 32) for this lane, summed by reduce_slots<S>.  TAB:
// C1s is the query's ADC table [256][M1] (FP16) and the term of code c is its entry [c][lane].
template <int M1, int D1, int S, typename CT, bool FQ, bool TAB = false>
__device__ __forceinline__ float score_slots(const CT *C1s, const uint8_t *stage, int nf, int d,
                                             const LaneGeo<M1, D1> &g, int lane, const CT *C2, int M2P)
{
    float v[S];
    if constexpr (TAB) {
        static_assert(M1 == 32 && !FQ, "the table form is built for 32 sub-spaces");
#pragma unroll
        for (int i = 0; i < S; i++) v[i] = i < nf ? to_f(C1s[(int)stage[i * M1 + lane] * M1 + lane]) : 0.f;
    } else if constexpr (FQ) {
        // full walk: one slot per step; the residual rows follow the 32 level-1 rows
        const uint8_t *stage2 = stage + 32 * M1;
        if (M1 == 16) {
            const int h = lane >> 4, j = lane & 15;
#pragma unroll
            for (int i = 0; i < S / 2; i++) {
                const int sl = 2 * i + h;
                float t = 0.f;
                if (2 * i < nf && sl < nf) t = part_full<M1, D1, CT>(C1s, C2, d, stage[sl * 16 + j], stage2 + sl * M2P, g, 0);
                v[2 * i] = h ? 0.f : t;
                v[2 * i + 1] = h ? t : 0.f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < S; i++) {
                float t = 0.f;
                if (i < nf) {
                    t = part_full<M1, D1, CT>(C1s, C2, d, stage[i * M1 + lane], stage2 + i * M2P, g, 0);
                    if (M1 == 64) t += part_full<M1, D1, CT>(C1s, C2, d, stage[i * M1 + 32 + lane], stage2 + i * M2P, g, 1);
                }
                v[i] = t;
            }
        }
    } else if (M1 == 16) {
        const int h = lane >> 4, j = lane & 15;
#pragma unroll
        for (int i = 0; i < S / 2; i++) {
            const int sl = 2 * i + h;                // half-warp h scores slots of parity h
            float t = 0.f;
            if (2 * i < nf && sl < nf) t = part_dist<M1, D1, CT>(C1s, d, stage[sl * 16 + j], g, 0);
            v[2 * i] = h ? 0.f : t;
            v[2 * i + 1] = h ? t : 0.f;
        }
    } else if (D1 > 0) {
        // two slots per step (the staged row of slot i + 1 >= nf is stale but a valid code;
        // its term is discarded)
#pragma unroll
        for (int i = 0; i < S; i += 2) {
            float t0 = 0.f, t1 = 0.f;
            if (i < nf) {
                pair_dist<M1, D1, CT>(C1s, d, stage[i * M1 + lane], stage[(i + 1) * M1 + lane], g, 0, t0, t1);
                if (M1 == 64) {
                    float u0, u1;
                    pair_dist<M1, D1, CT>(C1s, d, stage[i * M1 + 32 + lane], stage[(i + 1) * M1 + 32 + lane], g, 1, u0, u1);
                    t0 += u0;
                    t1 += u1;
                }
                if (i + 1 >= nf) t1 = 0.f;
            }
            v[i] = t0;
            v[i + 1] = t1;
        }
    } else {
#pragma unroll
        for (int i = 0; i < S; i++) {
            float t = 0.f;
            if (i < nf) {
                t = part_dist<M1, D1, CT>(C1s, d, stage[i * M1 + lane], g, 0);
                if (M1 == 64) t += part_dist<M1, D1, CT>(C1s, d, stage[i * M1 + 32 + lane], g, 1);
            }
            v[i] = t;
        }
    }
    return reduce_slots<S>(v, lane);
}

// Walk distances of the nf nodes in slot[0..nf) (1 <= nf <= 32): their code rows are staged
// in shared memory, each lane computes its sub-space terms, and the totals are formed with
// 16 or 32 slots.  Returns lane's total; *my_slot = the slot it holds (>= 32: none).
template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
__device__ __forceinline__ float score_nodes(const CT *C1s, uint8_t *stage, const uint8_t *codes1,
                                             const int32_t *slot, int nf, int d,
                                             const LaneGeo<M1, D1> &g, int lane, int *my_slot,
                                             const CT *C2, const uint8_t *codes2b, int M2P)
{
    if (lane < nf) {
        const uint4 *src = reinterpret_cast<const uint4 *>(codes1 + (int64_t)slot[lane] * M1);
        uint4 *dst = reinterpret_cast<uint4 *>(stage + lane * M1);
#pragma unroll
        for (int u = 0; u < M1 / 16; u++) dst[u] = __ldg(src + u);
        if constexpr (FQ) {
            const uint4 *s2 = reinterpret_cast<const uint4 *>(codes2b + (int64_t)slot[lane] * M2P);
            uint4 *d2 = reinterpret_cast<uint4 *>(stage + 32 * M1 + lane * M2P);
            for (int u = 0; u < M2P / 16; u++) d2[u] = __ldg(s2 + u);
        }
    }
    __syncwarp();
    float r;
    if (nf <= 16) {
        r = score_slots<M1, D1, 16, CT, FQ, TAB>(C1s, stage, nf, d, g, lane, C2, M2P);
        *my_slot = lane < 16 ? lane : 32;           // lanes l and l + 16 hold slot l
    } else {
        r = score_slots<M1, D1, 32, CT, FQ, TAB>(C1s, stage, nf, d, g, lane, C2, M2P);
        *my_slot = slot_of_lane(lane, 5);
    }
    __syncwarp();
    return r;
}

__device__ __forceinline__ uint32_t hash32(int32_t e)
{
    uint32_t x = (uint32_t)e * 0x9E3779B1u;
    return x ^ (x >> 15);
}

// Open addressing with triangular probing: the p-th probe of id e is at hash(e) + p(p+1)/2
// (mod the power-of-two table size), which visits every slot and, unlike a linear probe, does
// not grow long runs of occupied slots as the table fills (a warp resolves a row of 32 ids
// only when its longest probe sequence ends).
// Inserts e into the visited set; true if it was not there.  The shared table takes
// inserts until the walk switches to spill mode; from then on it is only read and new ids
// go to the warp's global table.
// Ids the shared visited table of H entries takes before the walk switches to the global one.
// Filling to three quarters rather than half (triangular probing: probe sequences stay short)
// measured 0.606 against 0.645 ms for the 1M workload's level-0 launch (fewer walks spill);
// seven eighths measured 0.654 ms.
__host__ __device__ constexpr int shared_visited_cap(int H) { return H - H / 4; }

__device__ __forceinline__ bool visit(int32_t e, int32_t *hash, int hlog, bool spilled,
                                      int32_t *spill, int slog)
{
    uint32_t Hm = (1u << hlog) - 1;
    uint32_t h = hash32(e) & Hm;
    if (!spilled) {
        for (uint32_t p = 0; p <= Hm; p++) {
            int32_t old = atomicCAS(hash + h, -1, e);
            if (old == -1) return true;
            if (old == e) return false;
            h = (h + p + 1) & Hm;
        }
        return false;   // unreachable: the table is kept at most three quarters full
    }
    for (uint32_t p = 0; p <= Hm; p++) {
        int32_t v = hash[h];
        if (v == e) return false;
        if (v == -1) break;
        h = (h + p + 1) & Hm;
    }
    uint32_t Sm = (1u << slog) - 1;
    h = (hash32(e) >> 3) & Sm;
    for (uint32_t p = 0; p <= Sm; p++) {
        int32_t old = atomicCAS(spill + h, -1, e);
        if (old == -1) return true;
        if (old == e) return false;
        h = (h + p + 1) & Sm;
    }
    return false;       // unreachable: the spill table is kept at most half full
}

// TAB (the table form, LC_LUT_TABLE): no codebook; each warp keeps its query's ADC table
// [256][M1] (FP16, built by table_kernel) in shared memory and scores nodes by table lookups.
template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
__global__ void __launch_bounds__(MAX_WALK_WARPS * 32) walk_kernel(const WalkArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d;
    // the level-1 codebook, shared by every warp of the CTA
    CT *C1s = reinterpret_cast<CT *>(smem_raw);
    if constexpr (!TAB) {
        const uint4 *src = reinterpret_cast<const uint4 *>(sizeof(CT) == 4 ? a.C1 : (const void *)a.C1h);
        uint4 *dst = reinterpret_cast<uint4 *>(C1s);
        const int n16 = (int)(walk_c1_bytes(d, M1, D1, sizeof(CT)) / 16);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    // full walk: C2 in shared memory (FP16) or read through the cache (FP32)
    const CT *C2 = nullptr;
    if constexpr (FQ) {
        if constexpr (sizeof(CT) == 2) {
            CT *C2s = reinterpret_cast<CT *>(smem_raw + walk_c1_bytes(d, M1, D1, sizeof(CT)));
            const uint4 *src = reinterpret_cast<const uint4 *>(a.C2h);
            for (int i = threadIdx.x; i < 256 * d * 2 / 16; i += blockDim.x) reinterpret_cast<uint4 *>(C2s)[i] = __ldg(src + i);
            C2 = C2s;
        } else {
            C2 = reinterpret_cast<const CT *>(a.C2);
        }
    }
    __syncthreads();
    const WalkSmem L = walk_smem(M1, d, a.efcap, a.hash_log, a.beam, a.yq_in == nullptr, FQ ? a.M2P : 0);
    constexpr size_t TABB = TAB ? (size_t)256 * M1 * 2 : 0;            // the query's table
    unsigned char *base = smem_raw + (TAB ? 0 : walk_cb_bytes(d, M1, D1, sizeof(CT), FQ)) + (size_t)warp * (L.total + TABB);
    if constexpr (TAB) C1s = reinterpret_cast<CT *>(base + L.total);
    float *yq = reinterpret_cast<float *>(base + L.yq);
    uint8_t *stage = base + L.stage;
    uint64_t *wkey = reinterpret_cast<uint64_t *>(base + L.wkey);
    uint8_t *wflag = base + L.wflag;
    uint64_t *cand = reinterpret_cast<uint64_t *>(base + L.cand);
    uint64_t *cuns = reinterpret_cast<uint64_t *>(base + L.cunsorted);
    int32_t *slot = reinterpret_cast<int32_t *>(base + L.slot);
    int32_t *rowbuf = reinterpret_cast<int32_t *>(base + L.rowbuf);
    int32_t *hash = reinterpret_cast<int32_t *>(base + L.hash);
    const int H = 1 << a.hash_log;
    const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int32_t *spill = a.spill + (gwarp << a.spill_log);
    const unsigned lt_mask = (1u << lane) - 1;

    for (;;) {
        int64_t qi = 0;
        if (lane == 0) qi = atomicAdd(a.counter, 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= a.nq) break;
        const int64_t q = a.order ? (int64_t)__ldg(a.order + qi) : qi;
        // this query's ef' = max(ef, k)
        const int efp = a.efq ? max(min(max(__ldg(a.efq + q), 1), a.efp), a.k) : a.efp;
        if constexpr (TAB) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.tab + q * 256 * M1);
            uint4 *dst = reinterpret_cast<uint4 *>(C1s);
#pragma unroll 4
            for (int i = lane; i < 256 * M1 * 2 / 16; i += 32) dst[i] = __ldg(src + i);
            __syncwarp();
        }
        // rotation y' = R y (fixed order u = 0..d-1); uint8 queries convert exactly to FP32
        const float *yrot = a.yq_in ? a.yq_in + q * d : yq;
        if (a.yq_in) {
            // computed by rotate_kernel
        } else if (a.Q8) {
            const uint8_t *y = a.Q8 + q * d;
            for (int t = lane; t < d; t += 32) {
                float s = 0.f;
                for (int u = 0; u < d; u++) s = fmaf(__ldg(a.Rt + (int64_t)u * d + t), (float)__ldg(y + u), s);
                yq[t] = s;
            }
        } else {
            const float *y = a.Q + q * d;
            for (int t = lane; t < d; t += 32) {
                float s = 0.f;
                for (int u = 0; u < d; u++) s = fmaf(__ldg(a.Rt + (int64_t)u * d + t), __ldg(y + u), s);
                yq[t] = s;
            }
        }
        if (a.mode != 1)
            for (int i = lane; i < H; i += 32) hash[i] = -1;
        __syncwarp();
        LaneGeo<M1, D1> g;
#pragma unroll
        for (int k = 0; k < LaneGeo<M1, D1>::NSUB; k++) {
            const int j = M1 == 16 ? (lane & 15) : lane + 32 * k;
            g.j[k] = j;
            g.off[k] = a.s1.off[j];
            g.len[k] = a.s1.len[j];
#pragma unroll
            for (int u = 0; u < LaneGeo<M1, D1>::DMAX; u++) {
                g.y[k][u] = u < g.len[k] ? yrot[g.off[k] + u] : 0.f;
                g.m2[k][u] = FQ && u < g.len[k] ? a.sub2[g.off[k] + u] : 0;
            }
        }
        int my_slot;
        // One loop runs the greedy descent of the upper levels (Section 2) and then the level-0
        // best-first search.  Each iteration gathers the nodes to score in slot[] and scores
        // them at a single call site, so the kernel holds one copy of the scoring code.
        int32_t n_up = 0, n_dist = 0, n_expand = 0;
        int32_t cur = a.ep;
        float dcur = 0.f;
        int lvl = a.max_level;             // upper level being descended
        int phase = 0;                     // 0: entry point, 1: upper levels, 2: level 0
        int wn = 1;
        bool spilled = false, failed = false;
        int32_t hcount = 1, scount = 0;
        int scan_from = 0;
        const int B = a.beam;              // level-0 expansions per step; 1 = the plain walk
        if (a.mode == 2) {
            // level 0 from the entry node the descent launch recorded (as at its end below)
            cur = __ldg(a.seed + q);
            dcur = __ldg(a.seed_d + q);
            n_up = __ldg(a.seed_up + q);
            phase = 2;
            if (lane == 0) {
                wkey[0] = make_key(dcur, cur);
                wflag[0] = 0;
                hash[hash32(cur) & (H - 1)] = cur;
            }
            n_dist = 1;
            __syncwarp();
        }
        for (;;) {
            uint64_t *W = wkey;
            uint8_t *F = wflag;
            int ns = 0, pos0 = 0;
            uint64_t ckey0 = 0;
            if (phase == 0) {
                if (lane == 0) slot[0] = cur;
                ns = 1;
            } else if (phase == 1) {
                // the current node's row at this level
                const int32_t e = a.upper_adj[((int64_t)a.upper_off[cur] + lvl - 1) * DEG + lane];
                const unsigned vm = __ballot_sync(FULL, e >= 0);
                ns = __popc(vm);
                if (e >= 0) slot[__popc(vm & lt_mask)] = e;
                n_up += ns;
            } else {
                if (a.tcap > 0 && n_dist >= a.tcap) break;     // search-time cap T (Section 3.1)
                // the B best unexpanded members of W: lane i < nb holds the i-th one's position
                int nb = 0, my_pos = -1;
                for (int b0 = scan_from; b0 < wn && nb < B; b0 += 32) {
                    const int p = b0 + lane;
                    unsigned m = __ballot_sync(FULL, p < wn && !F[p]);
                    while (m && nb < B) {
                        if (lane == nb) my_pos = b0 + __ffs(m) - 1;
                        nb++;
                        m &= m - 1;
                    }
                }
                if (nb == 0) break;
                pos0 = __shfl_sync(FULL, my_pos, 0);
                ckey0 = W[pos0];
                const int32_t my_c = lane < nb ? key_id(W[my_pos]) : -1;
                __syncwarp();
                if (lane < nb) F[my_pos] = 1;
                n_expand += nb;
                // their adjacency rows, all loads in flight together
                for (int r = 0; r < nb; r++) {
                    const int32_t cr = __shfl_sync(FULL, my_c, r);
                    rowbuf[r * DEG + lane] = a.adj0[(int64_t)cr * DEG + lane];
                }
                __syncwarp();
                // visited test row by row (row order, then slot order); fresh nodes are appended
                if (!spilled && hcount + 32 * nb <= shared_visited_cap(H)) {
                    // every row fits in the shared table without a switch to the spill table: the
                    // first probes of up to 4 rows are issued together, then each row is resolved
                    // in row order (a node in two rows probes the same bucket first, so it is
                    // fresh in the earlier row)
                    const uint32_t Hm = (uint32_t)H - 1;
                    for (int r0 = 0; r0 < nb; r0 += 4) {
                        int32_t ev[4], ov[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            ev[u] = r0 + u < nb ? rowbuf[(r0 + u) * DEG + lane] : -1;
                            ov[u] = ev[u] >= 0 ? atomicCAS(hash + (hash32(ev[u]) & Hm), -1, ev[u]) : 0;
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (r0 + u >= nb) break;
                            const int32_t e = ev[u];
                            bool fresh = e >= 0 && ov[u] == -1;
                            if (e >= 0 && ov[u] != -1 && ov[u] != e) {
                                // collision: continue the probe sequence
                                uint32_t h = hash32(e) & Hm;
                                for (uint32_t p = 1; p <= Hm; p++) {
                                    h = (h + p) & Hm;
                                    const int32_t old = atomicCAS(hash + h, -1, e);
                                    if (old == -1) { fresh = true; break; }
                                    if (old == e) break;
                                }
                            }
                            const unsigned fm = __ballot_sync(FULL, fresh);
                            if (fresh) slot[ns + __popc(fm & lt_mask)] = e;
                            const int nf = __popc(fm);
                            ns += nf;
                            n_dist += nf;
                            hcount += nf;
                        }
                    }
                } else if (spilled && scount + 32 * nb <= (1 << a.spill_log) / 2) {
                    // spilled, and every row fits in the global table: the shared table is only
                    // read; the first global probes of up to 4 rows are issued together, then
                    // each row is resolved in row order (as above)
                    const uint32_t Hm = (uint32_t)H - 1, Sm = (1u << a.spill_log) - 1;
                    for (int r0 = 0; r0 < nb; r0 += 4) {
                        int32_t ev[4], ov[4];
                        bool seen[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            ev[u] = r0 + u < nb ? rowbuf[(r0 + u) * DEG + lane] : -1;
                            seen[u] = false;
                            if (ev[u] >= 0) {
                                uint32_t h = hash32(ev[u]) & Hm;
                                for (uint32_t p = 0; p <= Hm; p++) {
                                    const int32_t v = hash[h];
                                    if (v == ev[u]) { seen[u] = true; break; }
                                    if (v == -1) break;
                                    h = (h + p + 1) & Hm;
                                }
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++)
                            ov[u] = ev[u] >= 0 && !seen[u] ? atomicCAS(spill + ((hash32(ev[u]) >> 3) & Sm), -1, ev[u]) : 0;
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (r0 + u >= nb) break;
                            const int32_t e = ev[u];
                            bool fresh = e >= 0 && !seen[u] && ov[u] == -1;
                            if (e >= 0 && !seen[u] && ov[u] != -1 && ov[u] != e) {
                                uint32_t h = (hash32(e) >> 3) & Sm;
                                for (uint32_t p = 1; p <= Sm; p++) {
                                    h = (h + p) & Sm;
                                    const int32_t old = atomicCAS(spill + h, -1, e);
                                    if (old == -1) { fresh = true; break; }
                                    if (old == e) break;
                                }
                            }
                            const unsigned fm = __ballot_sync(FULL, fresh);
                            if (fresh) slot[ns + __popc(fm & lt_mask)] = e;
                            const int nf = __popc(fm);
                            ns += nf;
                            n_dist += nf;
                            scount += nf;
                        }
                    }
                } else for (int r = 0; r < nb; r++) {
                    // switch to the global table before the shared one passes its limit
                    if (!spilled && hcount + 32 > shared_visited_cap(H)) {
                        spilled = true;
                        for (int i = lane; i < (1 << a.spill_log); i += 32) spill[i] = -1;
                        __syncwarp();
                    }
                    if (spilled && scount + 32 > (1 << a.spill_log) / 2) {
                        failed = true;
                        break;
                    }
                    const int32_t e = rowbuf[r * DEG + lane];
                    const bool fresh = e >= 0 && visit(e, hash, a.hash_log, spilled, spill, a.spill_log);
                    const unsigned fm = __ballot_sync(FULL, fresh);
                    if (fresh) slot[ns + __popc(fm & lt_mask)] = e;
                    const int nf = __popc(fm);
                    ns += nf;
                    n_dist += nf;
                    if (spilled) scount += nf; else hcount += nf;
                }
                if (failed) break;
                __syncwarp();
                if (ns == 0) { scan_from = pos0; continue; }
            }
            __syncwarp();
            // score the gathered nodes 32 at a time: the upper levels keep the best, level 0
            // keeps those that can enter W
            const uint64_t wmax = (phase == 2 && wn == efp) ? W[wn - 1] : ~0ull;
            uint64_t best = ~0ull;
            int nc = 0;
            for (int ch = 0; ch < ns; ch += 32) {
                const int nf = min(32, ns - ch);
                const float de = score_nodes<M1, D1, CT, FQ, TAB>(C1s, stage, a.codes1, slot + ch, nf, d, g, lane, &my_slot,
                                                             C2, a.codes2b, a.M2P);
                uint64_t k = my_slot < nf ? make_key(de, slot[ch + my_slot]) : ~0ull;
                if (phase < 2) {
                    best = warp_min64(k);                   // at most 32 nodes here
                } else {
                    if (k >= wmax) k = ~0ull;
                    const unsigned km = __ballot_sync(FULL, k != ~0ull);
                    if (k != ~0ull) cuns[nc + __popc(km & lt_mask)] = k;
                    nc += __popc(km);
                }
            }
            __syncwarp();
            if (phase < 2) {
                bool enter0 = false;
                if (phase == 0) {
                    dcur = key_dist(best);
                    if (lvl >= 1) {
                        n_up = 1;                           // the entry point's evaluation
                        phase = 1;
                    } else {
                        enter0 = true;
                    }
                } else if (ns > 0 && best < make_key(dcur, cur)) {
                    cur = key_id(best);                     // greedy move at this level
                    dcur = key_dist(best);
                } else if (--lvl == 0) {
                    enter0 = true;
                }
                if (enter0 && a.mode == 1) {
                    // descent only: record the level-0 entry for the second launch
                    if (lane == 0) {
                        a.seed[q] = cur;
                        a.seed_d[q] = dcur;
                        a.seed_up[q] = n_up;
                    }
                    break;
                }
                if (enter0) {
                    // level 0: best-first search with result list W (sorted keys + expanded flags)
                    phase = 2;
                    if (lane == 0) {
                        wkey[0] = make_key(dcur, cur);
                        wflag[0] = 0;
                        hash[hash32(cur) & (H - 1)] = cur;
                    }
                    n_dist = 1;
                    __syncwarp();
                }
                continue;
            }
            if (nc == 0) { scan_from = pos0; continue; }
            // order the candidates by rank (keys are distinct)
            for (int m0 = lane; m0 < nc; m0 += 32) {
                const uint64_t mk = cuns[m0];
                int r = 0;
                for (int m = 0; m < nc; m++) r += cuns[m] < mk;
                cand[r] = mk;
            }
            __syncwarp();
            // merge the nc candidates into W (wn keys) in place, keep ef': a candidate's place
            // is its rank plus the members below it, a member's its index plus the candidates
            // below it.  The candidates' places are taken first (into slot[], free after
            // scoring); members only move up, so chunks of 32 move from the last one down,
            // each read whole before it is written; the candidates are written last.
            const int wn2 = min(efp, wn + nc);
            int first_new = efp;
            for (int m0 = lane; m0 < nc; m0 += 32) {
                const uint64_t ck = cand[m0];
                int lo = 0, hi = wn;                     // W members below the candidate
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (W[mid] < ck) lo = mid + 1; else hi = mid;
                }
                slot[m0] = m0 + lo;
                if (m0 == 0) first_new = m0 + lo;
            }
            first_new = __shfl_sync(FULL, first_new, 0);
            __syncwarp();
            // members before the first candidate's place keep theirs
            for (int c0 = (wn - 1) & ~31; c0 >= (first_new & ~31); c0 -= 32) {
                const int p = c0 + lane;
                uint64_t key = 0;
                uint8_t f = 0;
                int np = p;
                if (p < wn) {
                    key = W[p];
                    f = F[p];
                    int lo = 0, hi = nc;                 // candidates below key
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cand[mid] < key) lo = mid + 1; else hi = mid;
                    }
                    np = p + lo;
                }
                __syncwarp();
                if (np != p && np < wn2) { W[np] = key; F[np] = f; }
                __syncwarp();
            }
            for (int m0 = lane; m0 < nc; m0 += 32) {
                const int np = slot[m0];
                if (np < wn2) { W[np] = cand[m0]; F[np] = 0; }
            }
            // everything before min(first new candidate, first expanded node's new place) is
            // expanded
            int below = 0;
            for (int m = 0; m < nc; m++) below += cand[m] < ckey0;
            scan_from = min(first_new, pos0 + below);
            scan_from -= scan_from % 32;
            wn = wn2;
            __syncwarp();
        }

        if (a.mode == 1) {
            __syncwarp();
            continue;
        }
        // outputs
        const uint64_t *W = wkey;
        if (a.refine) {
            if (!a.yq_in)
                for (int t = lane; t < d; t += 32) a.yq_out[q * d + t] = yq[t];
            for (int i = lane; i < a.R; i += 32)
                a.short_out[q * a.R + i] = (!failed && i < wn) ? key_id(W[i]) : -1;
        } else {
            for (int i = lane; i < a.R; i += 32) {
                bool ok = !failed && i < wn;
                a.ids_out[q * a.R + i] = ok ? key_id(W[i]) : -1;
                a.dists_out[q * a.R + i] = ok ? key_dist(W[i]) : __int_as_float(0x7f800000);
            }
        }
        if (lane == 0) {
            if (a.stats_out) {
                a.stats_out[q * 3 + 0] = failed ? -1 : n_dist;
                a.stats_out[q * 3 + 1] = n_expand;
                a.stats_out[q * 3 + 2] = n_up;
            }
            if (failed) atomicOr(a.status, 1);
        }
        __syncwarp();
    }
}


// ------------------------------------------------------------------------------------------
// Upper-level descent alone (the first launch of an ordered search): the greedy descent of
// Section 2 from the entry point down to level 1, exactly as walk_kernel runs it before level
// 0, writing each query's level-0 entry node, its walk distance and the upper-level
// evaluations.  It needs none of the level-0 state (result list, visited tables, merge
// buffers), so a warp holds only its staged code rows and node list: more warps fit per SM
// (up to 32), and more descents are in flight at once.
constexpr int MAX_DESCENT_WARPS = 32;

__host__ __device__ inline size_t descent_smem_per_warp(int M1, int m2p)
{
    return align_up((size_t)32 * (M1 + m2p), 16) + 32 * 4;
}

// threads per CTA the instantiation is compiled for: the full-decode walk keeps more per-lane
// state (the level-2 sub-space of every coordinate), so it gets registers for 16 warps
__host__ __device__ constexpr int descent_threads(bool fq) { return fq ? 16 * 32 : MAX_DESCENT_WARPS * 32; }

template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
__global__ void __launch_bounds__(descent_threads(FQ)) descent_kernel(const WalkArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d;
    CT *C1s = reinterpret_cast<CT *>(smem_raw);
    if constexpr (!TAB) {
        const uint4 *src = reinterpret_cast<const uint4 *>(sizeof(CT) == 4 ? a.C1 : (const void *)a.C1h);
        uint4 *dst = reinterpret_cast<uint4 *>(C1s);
        const int n16 = (int)(walk_c1_bytes(d, M1, D1, sizeof(CT)) / 16);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    const CT *C2 = nullptr;
    if constexpr (FQ) {
        if constexpr (sizeof(CT) == 2) {
            CT *C2s = reinterpret_cast<CT *>(smem_raw + walk_c1_bytes(d, M1, D1, sizeof(CT)));
            const uint4 *src = reinterpret_cast<const uint4 *>(a.C2h);
            for (int i = threadIdx.x; i < 256 * d * 2 / 16; i += blockDim.x) reinterpret_cast<uint4 *>(C2s)[i] = __ldg(src + i);
            C2 = C2s;
        } else {
            C2 = reinterpret_cast<const CT *>(a.C2);
        }
    }
    __syncthreads();
    const int m2p = FQ ? a.M2P : 0;
    unsigned char *base = smem_raw + (TAB ? 0 : walk_cb_bytes(d, M1, D1, sizeof(CT), FQ)) +
                          (size_t)warp * descent_smem_per_warp(M1, m2p);
    uint8_t *stage = base;
    int32_t *slot = reinterpret_cast<int32_t *>(base + align_up((size_t)32 * (M1 + m2p), 16));
    const unsigned lt_mask = (1u << lane) - 1;

    for (;;) {
        int64_t qi = 0;
        if (lane == 0) qi = atomicAdd(a.counter, 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= a.nq) break;
        const int64_t q = qi;
        const float *yrot = a.yq_in + q * d;       // y' = R y from the rotation kernel
        // TAB: the query's ADC table [256][M1], read through L1 (a descent scores few nodes)
        const CT *T1 = TAB ? reinterpret_cast<const CT *>(a.tab + q * 256 * M1) : C1s;
        LaneGeo<M1, D1> g;
#pragma unroll
        for (int k = 0; k < LaneGeo<M1, D1>::NSUB; k++) {
            const int j = M1 == 16 ? (lane & 15) : lane + 32 * k;
            g.j[k] = j;
            g.off[k] = a.s1.off[j];
            g.len[k] = a.s1.len[j];
#pragma unroll
            for (int u = 0; u < LaneGeo<M1, D1>::DMAX; u++) {
                g.y[k][u] = u < g.len[k] ? yrot[g.off[k] + u] : 0.f;
                g.m2[k][u] = FQ && u < g.len[k] ? a.sub2[g.off[k] + u] : 0;
            }
        }
        // the entry point's evaluation, then steepest moves level by level (as walk_kernel)
        int32_t cur = a.ep, n_up = 0;
        float dcur = 0.f;
        int lvl = a.max_level;
        bool first = true;
        for (;;) {
            int ns;
            if (first) {
                if (lane == 0) slot[0] = cur;
                ns = 1;
            } else {
                const int32_t e = a.upper_adj[((int64_t)a.upper_off[cur] + lvl - 1) * DEG + lane];
                const unsigned vm = __ballot_sync(FULL, e >= 0);
                ns = __popc(vm);
                if (e >= 0) slot[__popc(vm & lt_mask)] = e;
                n_up += ns;
            }
            __syncwarp();
            uint64_t best = ~0ull;
            if (ns > 0) {
                int my_slot;
                const float de = score_nodes<M1, D1, CT, FQ, TAB>(T1, stage, a.codes1, slot, ns, d, g, lane, &my_slot,
                                                                  C2, a.codes2b, a.M2P);
                const uint64_t k = my_slot < ns ? make_key(de, slot[my_slot]) : ~0ull;
                best = warp_min64(k);
            }
            __syncwarp();
            if (first) {
                first = false;
                dcur = key_dist(best);
                if (lvl < 1) break;
                n_up = 1;                                   // the entry point's evaluation
            } else if (ns > 0 && best < make_key(dcur, cur)) {
                cur = key_id(best);                         // greedy move at this level
                dcur = key_dist(best);
            } else if (--lvl == 0) {
                break;
            }
        }
        if (lane == 0) {
            a.seed[q] = cur;
            a.seed_d[q] = dcur;
            a.seed_up[q] = n_up;
        }
        __syncwarp();
    }
}

constexpr size_t MAX_SMEM_PER_BLOCK = 227 * 1024;

// Launch shape of the descent: as many warps as fit next to the codebook, at most 32.
template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
static cudaError_t launch_descent(const WalkArgs &wa, int sms, int *wpc_out, int *grid_out, size_t *smem_out)
{
    const size_t c1 = TAB ? 0 : walk_cb_bytes(wa.d, M1, D1, sizeof(CT), FQ);
    const size_t per = descent_smem_per_warp(M1, FQ ? wa.M2P : 0);
    if (c1 + per > MAX_SMEM_PER_BLOCK) return cudaErrorInvalidConfiguration;
    int wpc = (int)std::min<size_t>(MAX_DESCENT_WARPS, (MAX_SMEM_PER_BLOCK - c1) / per);
    cudaError_t e = cudaFuncSetAttribute(descent_kernel<M1, D1, CT, FQ, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MAX_SMEM_PER_BLOCK);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, descent_kernel<M1, D1, CT, FQ, TAB>);
    if (e != cudaSuccess) return e;
    wpc = std::min(wpc, fa.maxThreadsPerBlock / 32);
    const size_t smem = c1 + per * wpc;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, descent_kernel<M1, D1, CT, FQ, TAB>, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t need = (wa.nq + wpc - 1) / wpc;
    *grid_out = (int)std::min<int64_t>(need, (int64_t)per_sm * sms);
    *wpc_out = wpc;
    *smem_out = smem;
    return cudaSuccess;
}

// Compile-time shape of an instantiation (level-1 sub-quantisers, sub-space width, full walk),
// for dispatching a generic launcher over the instantiations.
template <int A, int B, bool C>
struct WalkShape {
    static constexpr int M1 = A, D1 = B;
    static constexpr bool FQ = C;
};

template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
static cudaError_t run_descent(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st)
{
    descent_kernel<M1, D1, CT, FQ, TAB><<<grid, wpc * 32, smem, st>>>(wa);
    return cudaGetLastError();
}

// Warps per CTA: as many as fit next to the codebook (at most MAX_WALK_WARPS, and at most
// want if want > 0).
template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
static cudaError_t launch_walk(const WalkArgs &wa, size_t smem_per_warp, int num_sms, int want, int *wpc_out,
                               int *grid_out, size_t *smem_out)
{
    size_t c1 = TAB ? 0 : walk_cb_bytes(wa.d, M1, D1, sizeof(CT), FQ);
    if (c1 + smem_per_warp > MAX_SMEM_PER_BLOCK) return cudaErrorInvalidConfiguration;
    int wpc = (int)std::min<size_t>(MAX_WALK_WARPS, (MAX_SMEM_PER_BLOCK - c1) / smem_per_warp);
    if (want > 0) wpc = std::min(wpc, want);
    size_t smem = c1 + smem_per_warp * wpc;
    // the attribute is an upper bound: set to the maximum, so plans made in any order (the
    // server plans at submission and launches later) all remain launchable
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<M1, D1, CT, FQ, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MAX_SMEM_PER_BLOCK);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<M1, D1, CT, FQ, TAB>, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (wa.nq + wpc - 1) / wpc;
    *grid_out = (int)std::min<int64_t>(need, (int64_t)per_sm * num_sms);
    *wpc_out = wpc;
    *smem_out = smem;
    return cudaSuccess;
}

template <int M1, int D1, typename CT, bool FQ, bool TAB = false>
static cudaError_t run_walk(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st)
{
    walk_kernel<M1, D1, CT, FQ, TAB><<<grid, wpc * 32, smem, st>>>(wa);
    return cudaGetLastError();
}


// Per element type (lc_walk_f32.cu, lc_walk_f16.cu): launch shape, launch and kernel address
// of the instantiation for a sub-space width variant, M1 and the full-decode flag.
cudaError_t walk_config_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms, int want,
                            int *wpc, int *grid, size_t *smem);
cudaError_t walk_run_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                         cudaStream_t st);
const void *walk_fn_f32(int variant, int M1, bool fq);
cudaError_t walk_config_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms, int want,
                            int *wpc, int *grid, size_t *smem);
cudaError_t walk_run_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                         cudaStream_t st);
const void *walk_fn_f16(int variant, int M1, bool fq);

cudaError_t descent_config_f32(int variant, int M1, bool fq, const WalkArgs &wa, int sms, int *wpc, int *grid,
                               size_t *smem);
cudaError_t descent_run_f32(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                            cudaStream_t st);
cudaError_t descent_config_f16(int variant, int M1, bool fq, const WalkArgs &wa, int sms, int *wpc, int *grid,
                               size_t *smem);
cudaError_t descent_run_f16(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                            cudaStream_t st);

inline cudaError_t descent_config(bool half, int variant, int M1, bool fq, const WalkArgs &wa, int sms, int *wpc,
                                  int *grid, size_t *smem)
{
    return half ? descent_config_f16(variant, M1, fq, wa, sms, wpc, grid, smem)
                : descent_config_f32(variant, M1, fq, wa, sms, wpc, grid, smem);
}
inline cudaError_t descent_run(bool half, int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc,
                               int grid, cudaStream_t st)
{
    return half ? descent_run_f16(variant, M1, fq, wa, smem, wpc, grid, st)
                : descent_run_f32(variant, M1, fq, wa, smem, wpc, grid, st);
}

// The table form (LC_LUT_TABLE; M1 = 32 at d = 96): launch shape, launch, kernel address of
// the walk, and the descent launch of an ordered search.
cudaError_t walk_config_tab(const WalkArgs &wa, size_t per_warp, int sms, int want, int *wpc, int *grid, size_t *smem);
cudaError_t walk_run_tab(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st);
const void *walk_fn_tab();
cudaError_t descent_config_tab(const WalkArgs &wa, int sms, int *wpc, int *grid, size_t *smem);
cudaError_t descent_run_tab(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st);

inline cudaError_t walk_config(bool half, int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms,
                               int want, int *wpc, int *grid, size_t *smem)
{
    return half ? walk_config_f16(variant, M1, fq, wa, per_warp, sms, want, wpc, grid, smem)
                : walk_config_f32(variant, M1, fq, wa, per_warp, sms, want, wpc, grid, smem);
}
inline cudaError_t walk_run(bool half, int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc,
                            int grid, cudaStream_t st)
{
    return half ? walk_run_f16(variant, M1, fq, wa, smem, wpc, grid, st)
                : walk_run_f32(variant, M1, fq, wa, smem, wpc, grid, st);
}
inline const void *walk_fn(bool half, int variant, int M1, bool fq)
{
    return half ? walk_fn_f16(variant, M1, fq) : walk_fn_f32(variant, M1, fq);
}

}  // namespace lc
