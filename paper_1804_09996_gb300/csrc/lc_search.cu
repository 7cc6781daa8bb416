// GPU search path of Link and Code (Douze, Sablayrolles, Jegou, CVPR 2018), sm_103a.
//
// walk_kernel  (one warp per query; persistent CTAs take queries from an atomic counter)
//   - rotation y' = R y; the walk distance is the ADC distance ||y' - c1(x)||^2 of Section
//     4.1 ("asymmetric distance computations"): the sum over level-1 sub-spaces j of
//     ||y'^j - C1_j[c_j]||^2, each term computed in FP32 from the codebook C1, which every
//     CTA keeps once in shared memory (a per-query table of the same terms would cost
//     32-64 KB of shared memory per query in flight);
//   - greedy descent of the upper HNSW levels (Section 2);
//   - best-first search of level 0 with result set W of size ef' (Section 2), kept as a
//     sorted list of (distance, id) keys with an "expanded" flag: each step expands the best
//     unexpanded member of W, scores all its unvisited neighbours at once (one per lane)
//     and merges them into W keeping the ef' best.  This expands exactly the nodes, in
//     exactly the order, of the two-set formulation (candidate heap C + result heap W);
//   - exact visited set: open-addressing hash in shared memory, spilling to a per-warp
//     table in global memory when it fills;
//   - writes the shortlist (the R best of W, Section 4.1 two-stage search) or, without
//     refinement, the top-k directly.
// refine_kernel (one warp per query)
//   - for each shortlisted x: G(x) = [q(x), q(g_1..g_8)] decoded from both code levels,
//     y^ = beta_b^T G(x) with b the vector's codeword (Section 4.3), exact squared L2 to
//     y', and the final top-k by (distance, id).
//
// FP32 walk distance: lane l holds the term of sub-space l (M1 = 32), of l mod 16 (M1 = 16)
// or the sum of sub-spaces l and l + 32 (M1 = 64), each term summed over its coordinates in
// order; the 32 lane values are added pairwise, lanes differing in bit 3 first, then bits 2,
// 1, 0 and 4.  The order is the same for every node, so a node's distance does not depend on
// where or with how many others it is scored.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lc_device.h"

namespace lc {

#define FULL 0xffffffffu

static void cfree(void *p) { if (p) cudaFree(p); }

void device_free(DeviceIndex *dv)
{
    if (!dv) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (dv->device >= 0) cudaSetDevice(dv->device);
    cfree(dv->Rt); cfree(dv->C1); cfree(dv->C2); cfree(dv->B); cfree(dv->C1h); cfree(dv->C1w); cfree(dv->C2h);
    cfree(dv->codes1); cfree(dv->codes2b);
    cfree(dv->adj0); cfree(dv->upper_off); cfree(dv->upper_adj);
    cfree(dv->yq); cfree(dv->shortlist); cfree(dv->spill); cfree(dv->status); cfree(dv->counter);
    cfree(dv->b_yq); cfree(dv->b_ids); cfree(dv->b_d); cfree(dv->b_rows); cfree(dv->b_idx); cfree(dv->b_sel);
    cfree(dv->q_st); cfree(dv->ef_st); cfree(dv->ids_st); cfree(dv->d_st); cfree(dv->s_st);
    for (auto &e : dv->ev) if (e) cudaEventDestroy(e);
    if (cur >= 0) cudaSetDevice(cur);
    delete dv;
}

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
// the rotation kernel's output.  The adjacency rows of a step are only read before the
// candidates are collected, so they share the unsorted-candidate area.
__host__ __device__ inline WalkSmem walk_smem(int M1, int d, int efcap, int hash_log, int beam, bool own_rot,
                                             int m2p = 0)
{
    WalkSmem s;
    size_t o = 0;
    s.yq = o;        o += own_rot ? align_up((size_t)d * 4, 16) : 0;
    s.stage = o;     o += (size_t)32 * (M1 + m2p);     // level-1 rows, then (full walk) residual rows
    s.wkey = o;      o += (size_t)2 * efcap * 8;
    s.wflag = o;     o += align_up((size_t)2 * efcap, 16);
    s.cand = o;      o += (size_t)32 * beam * 8;
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

// Sub-space terms of S slots (S = 16 or 32) for this lane, summed by reduce_slots<S>.
template <int M1, int D1, int S, typename CT, bool FQ>
__device__ __forceinline__ float score_slots(const CT *C1s, const uint8_t *stage, int nf, int d,
                                             const LaneGeo<M1, D1> &g, int lane, const CT *C2, int M2P)
{
    float v[S];
    if constexpr (FQ) {
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
template <int M1, int D1, typename CT, bool FQ>
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
        r = score_slots<M1, D1, 16, CT, FQ>(C1s, stage, nf, d, g, lane, C2, M2P);
        *my_slot = lane < 16 ? lane : 32;           // lanes l and l + 16 hold slot l
    } else {
        r = score_slots<M1, D1, 32, CT, FQ>(C1s, stage, nf, d, g, lane, C2, M2P);
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

// Inserts e into the visited set; true if it was not there.  The shared table takes
// inserts until the walk switches to spill mode; from then on it is only read and new ids
// go to the warp's global table.
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
            h = (h + 1) & Hm;
        }
        return false;   // unreachable: the table is kept at most half full
    }
    for (uint32_t p = 0; p <= Hm; p++) {
        int32_t v = hash[h];
        if (v == e) return false;
        if (v == -1) break;
        h = (h + 1) & Hm;
    }
    uint32_t Sm = (1u << slog) - 1;
    h = (hash32(e) >> 3) & Sm;
    for (uint32_t p = 0; p <= Sm; p++) {
        int32_t old = atomicCAS(spill + h, -1, e);
        if (old == -1) return true;
        if (old == e) return false;
        h = (h + 1) & Sm;
    }
    return false;       // unreachable: the spill table is kept at most half full
}

template <int M1, int D1, typename CT, bool FQ>
__global__ void __launch_bounds__(MAX_WALK_WARPS * 32) walk_kernel(const WalkArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d;
    // the level-1 codebook, shared by every warp of the CTA
    CT *C1s = reinterpret_cast<CT *>(smem_raw);
    {
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
    unsigned char *base = smem_raw + walk_cb_bytes(d, M1, D1, sizeof(CT), FQ) + (size_t)warp * L.total;
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
        int64_t q = 0;
        if (lane == 0) q = atomicAdd(a.counter, 1ull);
        q = __shfl_sync(FULL, q, 0);
        if (q >= a.nq) break;
        // this query's ef' = max(ef, k)
        const int efp = a.efq ? max(min(max(__ldg(a.efq + q), 1), a.efp), a.k) : a.efp;
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
        int buf = 0, wn = 1;
        bool spilled = false, failed = false;
        int32_t hcount = 1, scount = 0;
        int scan_from = 0;
        const int B = a.beam;              // level-0 expansions per step; 1 = the plain walk
        for (;;) {
            uint64_t *W = wkey + buf * a.efcap;
            uint8_t *F = wflag + buf * a.efcap;
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
                if (!spilled && hcount + 32 * nb <= H / 2) {
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
                                // collision: continue the linear probe
                                uint32_t h = hash32(e) & Hm;
                                for (uint32_t p = 1; p <= Hm; p++) {
                                    h = (h + 1) & Hm;
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
                                    h = (h + 1) & Hm;
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
                                    h = (h + 1) & Sm;
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
                    // switch to the global table before the shared one passes half full
                    if (!spilled && hcount + 32 > H / 2) {
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
                const float de = score_nodes<M1, D1, CT, FQ>(C1s, stage, a.codes1, slot + ch, nf, d, g, lane, &my_slot,
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
            // merge W (wn keys) with the nc candidates into the other buffer, keep ef'
            uint64_t *W2 = wkey + (buf ^ 1) * a.efcap;
            uint8_t *F2 = wflag + (buf ^ 1) * a.efcap;
            const int wn2 = min(efp, wn + nc);
            for (int p = lane; p < wn; p += 32) {
                const uint64_t key = W[p];
                int lo = 0, hi = nc;                     // candidates below key
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cand[mid] < key) lo = mid + 1; else hi = mid;
                }
                const int np = p + lo;
                if (np < wn2) { W2[np] = key; F2[np] = F[p]; }
            }
            int first_new = efp;
            for (int m0 = lane; m0 < nc; m0 += 32) {
                const uint64_t ck = cand[m0];
                int lo = 0, hi = wn;                     // W members below the candidate
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (W[mid] < ck) lo = mid + 1; else hi = mid;
                }
                const int np = m0 + lo;
                if (np < wn2) { W2[np] = ck; F2[np] = 0; }
                if (m0 == 0) first_new = np;
            }
            first_new = __shfl_sync(FULL, first_new, 0);
            // everything before min(first new candidate, first expanded node's new place) is
            // expanded
            int below = 0;
            for (int m = 0; m < nc; m++) below += cand[m] < ckey0;
            scan_from = min(first_new, pos0 + below);
            scan_from -= scan_from % 32;
            wn = wn2;
            buf ^= 1;
            __syncwarp();
        }

        // outputs
        const uint64_t *W = wkey + buf * a.efcap;
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
struct RefineArgs {
    const float *yq;
    const int32_t *shortlist;
    int64_t nq;
    int R, k, d, M1, M2P;           // M2P: padded row of the residual codes (codeword ids last)
    int BM, BK;                     // regression blocks, codewords per block (B: [BM][BK][9])
    const float *C1, *C2, *B;
    const uint8_t *codes1, *codes2b;
    const int32_t *adj0;
    int32_t *ids_out;
    float *dists_out;
    uint8_t sub1[256], sub2[256];   // sub-space of each dimension, per level
    uint8_t subb[256];              // regression block of each dimension
};

// ------------------------------------------------------------------------------------------
// Query rotation y' = R y (Section 3.3 / 5.1: OPQ rotates vectors and queries alike) for a
// whole batch ahead of the walk.  Every output coordinate is the fixed-order sum over
// u = 0..d-1 of R[t][u] y[u] (fmaf chain), the arithmetic of the walk's own rotation, so the
// walk gives bit-identical results either way.  R^T sits in shared memory when it fits
// (d <= 200); uint8 queries convert exactly to FP32.
constexpr int ROT_Q = 16;           // queries per block step (independent FMA chains per thread)
constexpr int ROT_THREADS = 128;
__host__ __device__ inline bool rotate_rt_shared(int d) { return (size_t)d * d * 4 <= 160 * 1024; }
__host__ __device__ inline size_t rotate_smem(int d)
{
    return ((rotate_rt_shared(d) ? (size_t)d * d : 0) + (size_t)ROT_Q * d) * 4;
}

// A thread owns output coordinate t of ROT_Q queries at a time: ROT_Q independent chains,
// with the queries' values read four at a time from ys [d][ROT_Q] (broadcast).
__global__ void __launch_bounds__(ROT_THREADS) rotate_kernel(const float *Q, const uint8_t *Q8, int64_t nq, int d,
                                                             const float *Rt, float *yq)
{
    extern __shared__ __align__(128) float rsm[];
    const bool shared_rt = rotate_rt_shared(d);
    float *ys = rsm + (shared_rt ? d * d : 0);
    const float *R = Rt;
    if (shared_rt) {
        // 16-byte loads, several in flight per thread (R^T is cudaMalloc-aligned)
        const int n4 = d * d / 4;
#pragma unroll 6
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            reinterpret_cast<float4 *>(rsm)[i] = __ldg(reinterpret_cast<const float4 *>(Rt) + i);
        for (int i = 4 * n4 + threadIdx.x; i < d * d; i += blockDim.x) rsm[i] = __ldg(Rt + i);
        R = rsm;
    }
    for (int64_t q0 = (int64_t)blockIdx.x * ROT_Q; q0 < nq; q0 += (int64_t)gridDim.x * ROT_Q) {
        const int nb = nq - q0 < ROT_Q ? (int)(nq - q0) : ROT_Q;
        __syncthreads();                               // Rt loaded / previous step's ys consumed
#pragma unroll 4
        for (int i = threadIdx.x; i < ROT_Q * d; i += blockDim.x) {
            const int qq = i / d, u = i - qq * d;
            ys[u * ROT_Q + qq] = qq >= nb ? 0.f : Q8 ? (float)__ldg(Q8 + (q0 + qq) * d + u) : __ldg(Q + (q0 + qq) * d + u);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < d; t += blockDim.x) {
            float acc[ROT_Q];
#pragma unroll
            for (int qq = 0; qq < ROT_Q; qq++) acc[qq] = 0.f;
#pragma unroll 4
            for (int u = 0; u < d; u++) {
                const float r = R[u * d + t];
                const float4 *y4 = reinterpret_cast<const float4 *>(ys + u * ROT_Q);
#pragma unroll
                for (int v = 0; v < ROT_Q / 4; v++) {
                    const float4 y = y4[v];
                    acc[4 * v + 0] = fmaf(r, y.x, acc[4 * v + 0]);
                    acc[4 * v + 1] = fmaf(r, y.y, acc[4 * v + 1]);
                    acc[4 * v + 2] = fmaf(r, y.z, acc[4 * v + 2]);
                    acc[4 * v + 3] = fmaf(r, y.w, acc[4 * v + 3]);
                }
            }
#pragma unroll
            for (int qq = 0; qq < ROT_Q; qq++)
                if (qq < nb) yq[(q0 + qq) * d + t] = acc[qq];
        }
    }
}

constexpr int REF_CH = 8;            // candidates staged at a time

__host__ __device__ inline int pow2_at_least(int r)
{
    int p = 32;
    while (p < r) p <<= 1;
    return p;
}

// Per-warp shared memory of the refinement kernel.
__host__ __device__ inline size_t refine_smem(int M1, int M2P, int R, int BM)
{
    size_t o = 0;
    o += (size_t)REF_CH * 9 * 4;            // vertex ids
    o += (size_t)REF_CH * 9 * 4 * BM;       // weights, per regression block
    o = align_up(o, 16);                    // code rows are written 16 bytes at a time
    o += (size_t)REF_CH * 9 * M1;           // level-1 code rows
    o += (size_t)REF_CH * 9 * M2P;          // level-2 code rows (+ codeword id)
    o += (size_t)pow2_at_least(R) * 8;      // keys
    return align_up(o, 128);
}

// One warp per query.  C2_SHARED: both codebooks sit in shared memory (d*4 bytes is a
// multiple of 128, so lane t reading coordinate t of any centroid hits bank t mod 32);
// otherwise only C1 does and C2 is read through the cache.  DU: coordinates per lane
// (d = 32 DU), or 8 with bounds checks for other d <= 256.
template <bool C2_SHARED, int DU, bool PROD>
__global__ void __launch_bounds__(16 * 32) refine_kernel(const RefineArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, M1 = a.M1, M2P = a.M2P;
    float *C1s = reinterpret_cast<float *>(smem_raw);
    float *C2s = C1s + 256 * d;
    {
        const float4 *s1 = reinterpret_cast<const float4 *>(a.C1);
        const float4 *s2 = reinterpret_cast<const float4 *>(a.C2);
        for (int i = threadIdx.x; i < 64 * d; i += blockDim.x) {
            reinterpret_cast<float4 *>(C1s)[i] = __ldg(s1 + i);
            if (C2_SHARED) reinterpret_cast<float4 *>(C2s)[i] = __ldg(s2 + i);
        }
    }
    __syncthreads();
    const float *C2 = C2_SHARED ? C2s : a.C2;
    const size_t cb = (size_t)(C2_SHARED ? 2 : 1) * 256 * d * 4;
    const int BM = PROD ? a.BM : 1;
    unsigned char *base = smem_raw + cb + (size_t)warp * refine_smem(M1, M2P, a.R, BM);
    const int RP = pow2_at_least(a.R);
    int32_t *vid = reinterpret_cast<int32_t *>(base);
    float *wt = reinterpret_cast<float *>(base + REF_CH * 9 * 4);       // [REF_CH][BM][9]
    uint8_t *st1 = base + align_up((size_t)REF_CH * 9 * 4 * (1 + BM), 16);
    uint8_t *st2 = st1 + REF_CH * 9 * M1;
    uint64_t *keys = reinterpret_cast<uint64_t *>(st2 + REF_CH * 9 * M2P);
    const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int r1 = M1 / 16, r2 = M2P / 16;          // 16-byte pieces per row
    // sub-spaces of this lane's coordinates t = lane + 32 u (read once: indexing the
    // parameter space with a per-lane index would serialise)
    int s1v[DU], s2v[DU], sbv[DU];
#pragma unroll
    for (int u = 0; u < DU; u++) {
        const int t = lane + 32 * u;
        s1v[u] = t < d ? a.sub1[t] : 0;
        s2v[u] = t < d ? a.sub2[t] : 0;
        sbv[u] = PROD && t < d ? a.subb[t] : 0;
    }
    const int nb = a.BK > 1 ? BM : 0;               // codeword bytes at the end of a row

    for (int64_t q = gwarp; q < a.nq; q += nwarps) {
        const int32_t *sl = a.shortlist + q * a.R;
        float yv[DU];
#pragma unroll
        for (int u = 0; u < DU; u++) yv[u] = lane + 32 * u < d ? a.yq[q * d + lane + 32 * u] : 0.f;
        int rn = 0;                                  // shortlist entries present (packed first)
        for (int i = lane; i < a.R; i += 32) rn += sl[i] >= 0;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) rn += __shfl_xor_sync(FULL, rn, m);
        for (int i = lane; i < RP; i += 32) keys[i] = ~0ull;
        for (int c0 = 0; c0 < rn; c0 += REF_CH) {
            const int nc = min(REF_CH, rn - c0);
            // one candidate per lane: its id, codeword and the 8 neighbours of G(x); the
            // loads of a phase are all issued before any is used
            if (lane < nc) {
                const int32_t i = sl[c0 + lane];
                const uint8_t *crow = a.codes2b + (int64_t)i * M2P + M2P - nb;
                const int4 *ar = reinterpret_cast<const int4 *>(a.adj0 + (int64_t)i * DEG);
                const int4 a0 = __ldg(ar), a1 = __ldg(ar + 1);
                int32_t *vr = vid + lane * 9;
                vr[0] = i;
                vr[1] = a0.x; vr[2] = a0.y; vr[3] = a0.z; vr[4] = a0.w;
                vr[5] = a1.x; vr[6] = a1.y; vr[7] = a1.z; vr[8] = a1.w;
                for (int m = 0; m < BM; m++) {
                    const int b = nb ? crow[m] : 0;
                    const float *bw = a.B + ((int64_t)m * a.BK + b) * 9;
                    float w[9];
#pragma unroll
                    for (int j = 0; j < 9; j++) w[j] = __ldg(bw + j);
#pragma unroll
                    for (int j = 0; j < 9; j++) wt[(lane * BM + m) * 9 + j] = w[j];
                }
            }
            __syncwarp();
            // stage both code rows of every vertex: 16-byte pieces, six loads in flight per lane
            const int per_row = r1 + r2, pieces = nc * 9 * per_row;
            for (int t0 = lane; t0 < pieces; t0 += 32 * 6) {
                uint4 buf[6];
                bool use[6];
#pragma unroll
                for (int u = 0; u < 6; u++) {
                    const int t = t0 + 32 * u;
                    const int row = t / per_row, pc = t % per_row;
                    use[u] = t < pieces && vid[row] >= 0;
                    if (use[u]) {
                        const int64_t v = vid[row];
                        buf[u] = pc < r1 ? __ldg(reinterpret_cast<const uint4 *>(a.codes1 + v * M1) + pc)
                                         : __ldg(reinterpret_cast<const uint4 *>(a.codes2b + v * M2P) + (pc - r1));
                    }
                }
#pragma unroll
                for (int u = 0; u < 6; u++) {
                    const int t = t0 + 32 * u;
                    const int row = t / per_row, pc = t % per_row;
                    if (use[u]) {
                        if (pc < r1) reinterpret_cast<uint4 *>(st1 + row * M1)[pc] = buf[u];
                        else reinterpret_cast<uint4 *>(st2 + row * M2P)[pc - r1] = buf[u];
                    }
                }
            }
            __syncwarp();
            for (int r = 0; r < nc; r++) {
                // y^_t = sum_j beta_j (C1[c1_j][t] + C2[c2_j][t]) for this lane's coordinates,
                // accumulated over j in order; then sum_t (y'_t - y^_t)^2 over t ascending
                float yh[DU];
#pragma unroll
                for (int u = 0; u < DU; u++) yh[u] = 0.f;
#pragma unroll
                for (int j = 0; j < 9; j++) {
                    const int tt = r * 9 + j;
                    if (vid[tt] < 0) continue;
                    const float w0 = wt[r * BM * 9 + j];
                    const uint8_t *c1r = st1 + tt * M1, *c2r = st2 + tt * M2P;
#pragma unroll
                    for (int u = 0; u < DU; u++) {
                        const int t = lane + 32 * u;
                        if (DU == 8 && t >= d) continue;
                        // the weight of this coordinate's regression block
                        const float w = PROD ? wt[(r * BM + sbv[u]) * 9 + j] : w0;
                        const float x = C1s[(int)c1r[s1v[u]] * d + t] + C2[(int)c2r[s2v[u]] * d + t];
                        yh[u] = fmaf(w, x, yh[u]);
                    }
                }
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < DU; u++) {
                    if (DU == 8 && lane + 32 * u >= d) continue;
                    const float df = yv[u] - yh[u];
                    part = fmaf(df, df, part);
                }
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) part += __shfl_xor_sync(FULL, part, m);
                if (lane == 0) keys[c0 + r] = make_key(part, vid[r * 9]);
            }
            __syncwarp();
        }
        __syncwarp();
        // bitonic sort of keys[0..RP) ascending
        for (int kk = 2; kk <= RP; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < RP; i += 32) {
                    int p = i ^ j;
                    if (p > i) {
                        uint64_t x = keys[i], y = keys[p];
                        bool up = (i & kk) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[p] = x; }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < a.k; i += 32) {
            uint64_t kk = keys[i];
            bool ok = kk != ~0ull;
            a.ids_out[q * a.k + i] = ok ? key_id(kk) : -1;
            a.dists_out[q * a.k + i] = ok ? key_dist(kk) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Host side
template <class T>
static bool dupload(T *&dst, const std::vector<T> &src)
{
    cfree(dst);
    dst = nullptr;
    size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
    if (cudaMalloc(&dst, bytes) != cudaSuccess) return false;
    if (!src.empty() && cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    return true;
}

template <class T>
static bool grow(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return true;
    cfree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) return false;
    cap = need;
    return true;
}

lc_status upload(lc_index *ix)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    if (ix->dev && (!ix->dev_dirty && ix->dev->device == dev)) return LC_OK;
    DeviceIndex *dv = ix->dev;
    if (dv && dv->device != dev) {
        device_free(dv);
        dv = ix->dev = nullptr;
    }
    if (!dv) {
        dv = ix->dev = new DeviceIndex();
        dv->device = dev;
        cudaDeviceGetAttribute(&dv->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaMalloc(&dv->status, sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&dv->counter, sizeof(unsigned long long)) != cudaSuccess) {
            set_error("cudaMalloc failed for the status word");
            return LC_ERR_OOM;
        }
    }
    int d = ix->p.d;
    std::vector<float> Rt((size_t)d * d);
    for (int t = 0; t < d; t++)
        for (int u = 0; u < d; u++) Rt[(size_t)u * d + t] = ix->R[(size_t)t * d + u];
    std::vector<int32_t> off(ix->n);
    for (int64_t i = 0; i < ix->n; i++) off[i] = (int32_t)ix->upper_off[i];
    // residual codes, then the regression codeword ids (one per block; none with the
    // 0-byte weights) in the last bytes of a 16-byte-aligned row
    const int M2 = ix->p.M2, bM = ix->p.beta_M, bK = ix->p.beta_K;
    const int nb = bK > 1 ? bM : 0;
    const int M2P = (int)align_up((size_t)M2 + nb, 16);
    std::vector<uint8_t> c2b((size_t)ix->n * M2P, 0);
    for (int64_t i = 0; i < ix->n; i++) {
        std::memcpy(c2b.data() + i * M2P, ix->codes2.data() + i * M2, M2);
        for (int m = 0; m < nb; m++) c2b[i * M2P + M2P - nb + m] = ix->beta[i * bM + m];
    }
    // the walk's level-1 codebook, FP32 and FP16 (rounded to nearest even), in its layout
    const int M1 = ix->p.M1, D1 = walk_variant_d1(walk_variant(M1, d));
    std::vector<int> so, sl;
    splits(d, M1, so, sl);
    auto put_layout = [&](int es, auto put) {
        const int L = walk_layout(D1, es), P = walk_pad(D1);
        for (int c = 0; c < 256; c++)
            for (int j = 0; j < M1; j++)
                for (int u = 0; u < sl[j]; u++) {
                    const float v = ix->C1[(size_t)c * d + so[j] + u];
                    if (L == 0) put((size_t)c * d + so[j] + u, v);
                    else if (L == 1) put(((size_t)c * M1 + j) * P + u, v);
                    else put(u < 2 ? ((size_t)c * M1 + j) * 2 + u : (size_t)256 * M1 * 2 + (size_t)c * M1 + j, v);
                }
    };
    std::vector<float> c1w(walk_c1_bytes(d, M1, D1, 4) / 4, 0.f);
    put_layout(4, [&](size_t i, float v) { c1w[i] = v; });
    std::vector<__half> c1h(walk_c1_bytes(d, M1, D1, 2) / 2, __float2half_rn(0.f));
    put_layout(2, [&](size_t i, float v) { c1h[i] = __float2half_rn(v); });
    std::vector<__half> c2h(ix->C2.size());
    for (size_t i = 0; i < c2h.size(); i++) c2h[i] = __float2half_rn(ix->C2[i]);   // round to nearest even
    __half *c2h_dev = static_cast<__half *>(dv->C2h);
    __half *c1h_dev = static_cast<__half *>(dv->C1h);
    bool ok = dupload(dv->Rt, Rt) && dupload(dv->C1, ix->C1) && dupload(dv->C2, ix->C2) &&
              dupload(dv->C1w, c1w) && dupload(c1h_dev, c1h) && dupload(c2h_dev, c2h) &&
              dupload(dv->B, ix->B) && dupload(dv->codes1, ix->codes1) &&
              dupload(dv->codes2b, c2b) &&
              dupload(dv->adj0, ix->adj0) && dupload(dv->upper_off, off) &&
              dupload(dv->upper_adj, ix->upper_adj);
    dv->C1h = c1h_dev;
    dv->C2h = c2h_dev;
    if (!ok) {
        set_error("device upload of the index failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_OOM;
    }
    dv->n = ix->n;
    dv->d = d;
    dv->M1 = ix->p.M1;
    dv->M2 = ix->p.M2;
    dv->M2P = M2P;
    dv->bM = bM;
    dv->bK = bK;
    dv->ep = ix->ep;
    dv->max_level = ix->max_level < 0 ? 0 : ix->max_level;
    static std::atomic<uint64_t> uploads{0};
    dv->gen = ++uploads;
    ix->dev_dirty = false;
    return LC_OK;
}

static int ilog2_ceil(int64_t x)
{
    int l = 0;
    while (((int64_t)1 << l) < x) l++;
    return l;
}

constexpr size_t MAX_SMEM_PER_BLOCK = 227 * 1024;

// Warps per CTA: as many as fit next to the codebook (at most MAX_WALK_WARPS, and at most
// want if want > 0).
template <int M1, int D1, typename CT, bool FQ>
static cudaError_t launch_walk(const WalkArgs &wa, size_t smem_per_warp, int num_sms, int want, int *wpc_out,
                               int *grid_out, size_t *smem_out)
{
    size_t c1 = walk_cb_bytes(wa.d, M1, D1, sizeof(CT), FQ);
    if (c1 + smem_per_warp > MAX_SMEM_PER_BLOCK) return cudaErrorInvalidConfiguration;
    int wpc = (int)std::min<size_t>(MAX_WALK_WARPS, (MAX_SMEM_PER_BLOCK - c1) / smem_per_warp);
    if (want > 0) wpc = std::min(wpc, want);
    size_t smem = c1 + smem_per_warp * wpc;
    // the attribute is an upper bound: set to the maximum, so plans made in any order (the
    // server plans at submission and launches later) all remain launchable
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<M1, D1, CT, FQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MAX_SMEM_PER_BLOCK);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<M1, D1, CT, FQ>, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (wa.nq + wpc - 1) / wpc;
    *grid_out = (int)std::min<int64_t>(need, (int64_t)per_sm * num_sms);
    *wpc_out = wpc;
    *smem_out = smem;
    return cudaSuccess;
}

template <int M1, int D1, typename CT, bool FQ>
static cudaError_t run_walk(const WalkArgs &wa, size_t smem, int wpc, int grid, cudaStream_t st)
{
    walk_kernel<M1, D1, CT, FQ><<<grid, wpc * 32, smem, st>>>(wa);
    return cudaGetLastError();
}

using RefineFn = void (*)(const RefineArgs);

// Refinement instantiation: codebooks placement and coordinates per lane (3 for d = 96,
// 4 for d = 128, else the checked 8).
static RefineFn refine_kernel_for(bool both, int d, bool prod)
{
    if (prod) {
        if (d == 96) return both ? refine_kernel<true, 3, true> : refine_kernel<false, 3, true>;
        if (d == 128) return both ? refine_kernel<true, 4, true> : refine_kernel<false, 4, true>;
        return both ? refine_kernel<true, 8, true> : refine_kernel<false, 8, true>;
    }
    if (d == 96) return both ? refine_kernel<true, 3, false> : refine_kernel<false, 3, false>;
    if (d == 128) return both ? refine_kernel<true, 4, false> : refine_kernel<false, 4, false>;
    return both ? refine_kernel<true, 8, false> : refine_kernel<false, 8, false>;
}

// Dispatch on (sub-space width variant, codebook element type, full walk).  The full walk
// exists for the uniform splits (variants 1-3) and, in FP32, for any split.
template <typename CT>
static cudaError_t launch_any(int variant, int M1, bool fq, const WalkArgs &wa, size_t per_warp, int sms, int want,
                              int *wpc, int *grid, size_t *smem)
{
    if (fq) {
        switch (variant) {
        case 1: return launch_walk<16, 6, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 2: return launch_walk<32, 3, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
        case 3: return launch_walk<64, 2, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
        default:
            if constexpr (sizeof(CT) == 4) {
                if (M1 == 16) return launch_walk<16, 0, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
                if (M1 == 32) return launch_walk<32, 0, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
                return launch_walk<64, 0, CT, true>(wa, per_warp, sms, want, wpc, grid, smem);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return launch_walk<16, 6, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 2: return launch_walk<32, 3, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
    case 3: return launch_walk<64, 2, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
    default:
        if (M1 == 16) return launch_walk<16, 0, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
        if (M1 == 32) return launch_walk<32, 0, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
        return launch_walk<64, 0, CT, false>(wa, per_warp, sms, want, wpc, grid, smem);
    }
}

// The walk instantiation a plan launches (for finding its node in a captured graph).
template <typename CT>
static const void *walk_fn(int variant, int M1, bool fq)
{
    if (fq) {
        switch (variant) {
        case 1: return (const void *)walk_kernel<16, 6, CT, true>;
        case 2: return (const void *)walk_kernel<32, 3, CT, true>;
        case 3: return (const void *)walk_kernel<64, 2, CT, true>;
        default:
            if constexpr (sizeof(CT) == 4) {
                if (M1 == 16) return (const void *)walk_kernel<16, 0, CT, true>;
                if (M1 == 32) return (const void *)walk_kernel<32, 0, CT, true>;
                return (const void *)walk_kernel<64, 0, CT, true>;
            }
            return nullptr;
        }
    }
    switch (variant) {
    case 1: return (const void *)walk_kernel<16, 6, CT, false>;
    case 2: return (const void *)walk_kernel<32, 3, CT, false>;
    case 3: return (const void *)walk_kernel<64, 2, CT, false>;
    default:
        if (M1 == 16) return (const void *)walk_kernel<16, 0, CT, false>;
        if (M1 == 32) return (const void *)walk_kernel<32, 0, CT, false>;
        return (const void *)walk_kernel<64, 0, CT, false>;
    }
}

template <typename CT>
static cudaError_t run_any(int variant, int M1, bool fq, const WalkArgs &wa, size_t smem, int wpc, int grid,
                           cudaStream_t st)
{
    if (fq) {
        switch (variant) {
        case 1: return run_walk<16, 6, CT, true>(wa, smem, wpc, grid, st);
        case 2: return run_walk<32, 3, CT, true>(wa, smem, wpc, grid, st);
        case 3: return run_walk<64, 2, CT, true>(wa, smem, wpc, grid, st);
        default:
            if constexpr (sizeof(CT) == 4) {
                if (M1 == 16) return run_walk<16, 0, CT, true>(wa, smem, wpc, grid, st);
                if (M1 == 32) return run_walk<32, 0, CT, true>(wa, smem, wpc, grid, st);
                return run_walk<64, 0, CT, true>(wa, smem, wpc, grid, st);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
    case 1: return run_walk<16, 6, CT, false>(wa, smem, wpc, grid, st);
    case 2: return run_walk<32, 3, CT, false>(wa, smem, wpc, grid, st);
    case 3: return run_walk<64, 2, CT, false>(wa, smem, wpc, grid, st);
    default:
        if (M1 == 16) return run_walk<16, 0, CT, false>(wa, smem, wpc, grid, st);
        if (M1 == 32) return run_walk<32, 0, CT, false>(wa, smem, wpc, grid, st);
        return run_walk<64, 0, CT, false>(wa, smem, wpc, grid, st);
    }
}

lc_status plan_search(const DeviceIndex *dv, int64_t nq, const lc_search_params *sp, SearchPlan *pl)
{
    SearchPlan P;
    P.k = sp->k;
    P.efp = std::max(sp->ef, sp->k);
    P.refine = sp->shortlist >= 0;
    P.R = P.refine ? std::max(sp->shortlist > 0 ? sp->shortlist : 10, P.k) : P.k;
    if (P.refine && P.R > MAX_SHORTLIST) {
        set_error("shortlist %d exceeds %d", P.R, MAX_SHORTLIST);
        return LC_ERR_ARG;
    }
    P.beam = sp->mode == LC_MODE_BATCHED ? sp->beam : 1;
    P.tcap = sp->max_dist;
    P.hash_log = sp->visited_log ? sp->visited_log : std::min(12, std::max(10, ilog2_ceil((int64_t)P.efp * 32)));
    P.spill_log = std::min(16, std::max(13, ilog2_ceil((int64_t)P.efp * 64)));
    const int efcap = (int)align_up(P.efp, 32);
    // compile-time sub-space width for the uniform splits 96/16, 96/32, 128/64
    P.variant = walk_variant(dv->M1, dv->d);
    P.full = sp->walk_full != 0;
    if (P.full && P.variant == 0 && sp->lut_prec == LC_LUT_FP16) {
        set_error("the full-decode walk in FP16 needs a uniform level-1 split (M1 = 16 or 32 at d = 96, "
                  "M1 = 64 at d = 128); use FP32");
        return LC_ERR_ARG;
    }
    P.per_warp = walk_smem(dv->M1, dv->d, efcap, P.hash_log, P.beam, false, P.full ? dv->M2P : 0).total;
    WalkArgs wa{};
    wa.nq = nq;
    wa.d = dv->d;
    P.half = sp->lut_prec == LC_LUT_FP16;
    cudaError_t ce = P.half ? launch_any<__half>(P.variant, dv->M1, P.full, wa, P.per_warp, dv->num_sms, sp->warps, &P.wpc, &P.grid, &P.smem)
                            : launch_any<float>(P.variant, dv->M1, P.full, wa, P.per_warp, dv->num_sms, sp->warps, &P.wpc, &P.grid, &P.smem);
    if (ce == cudaErrorInvalidConfiguration) {
        set_error("search too wide for shared memory (%zu B per query in flight next to a %zu B codebook); "
                  "lower efSearch or visited_log", P.per_warp,
                  walk_cb_bytes(dv->d, dv->M1, walk_variant_d1(P.variant), P.half ? 2 : 4, P.full));
        return LC_ERR_CAPACITY;
    }
    if (ce != cudaSuccess) {
        set_error("walk kernel configuration failed (%zu B shared memory per warp): %s", P.per_warp,
                  cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    P.spill_elems = ((size_t)P.grid * P.wpc) << P.spill_log;
    P.yq_elems = (size_t)nq * dv->d;
    {
        const size_t rsm = rotate_smem(dv->d);
        if (cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_SMEM_PER_BLOCK) != cudaSuccess) {
            set_error("rotation kernel configuration failed: %s", cudaGetErrorString(cudaGetLastError()));
            return LC_ERR_CUDA;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rotate_kernel, ROT_THREADS, rsm);
        P.qsm = rsm;
        // as many blocks as fit at once: the batch is rotated in about one step per block
        P.qgrid = (int)std::min<int64_t>((nq + ROT_Q - 1) / ROT_Q, (int64_t)std::max(per_sm, 1) * dv->num_sms);
    }
    if (P.refine) {
        P.sl_elems = (size_t)nq * P.R;
        const size_t per = refine_smem(dv->M1, dv->M2P, P.R, dv->bM);
        const size_t cbytes = (size_t)256 * dv->d * 4;
        // both codebooks in shared memory when that leaves room for at least 8 warps
        P.rboth = 2 * cbytes + 8 * per <= MAX_SMEM_PER_BLOCK;
        const size_t cb = (P.rboth ? 2 : 1) * cbytes;
        if (cb + per > MAX_SMEM_PER_BLOCK) {
            set_error("refinement does not fit in shared memory (d = %d)", dv->d);
            return LC_ERR_CAPACITY;
        }
        P.rw = (int)std::min<size_t>(16, (MAX_SMEM_PER_BLOCK - cb) / per);
        P.rsm = cb + per * P.rw;
        auto kern = refine_kernel_for(P.rboth, dv->d, dv->bM > 1);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_SMEM_PER_BLOCK) != cudaSuccess) {
            set_error("refine kernel configuration failed: %s", cudaGetErrorString(cudaGetLastError()));
            return LC_ERR_CUDA;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P.rw * 32, P.rsm);
        const int64_t need = (nq + P.rw - 1) / P.rw;
        P.rgrid = (int)std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * dv->num_sms);
    }
    *pl = P;
    return LC_OK;
}

lc_status run_search(DeviceIndex *dv, const SearchPlan &P, const float *dq, int64_t nq, int32_t *dids,
                     float *ddists, int32_t *dstats, const SearchScratch &sc, cudaStream_t st, bool profile,
                     const uint8_t *dq8, const int32_t *defq, bool rotated)
{
    WalkArgs wa{};
    wa.Q = dq; wa.Q8 = dq8; wa.efq = defq; wa.k = P.k; wa.nq = nq; wa.d = dv->d;
    wa.Rt = dv->Rt; wa.C1 = dv->C1w; wa.C1h = static_cast<const __half *>(dv->C1h); wa.codes1 = dv->codes1;
    wa.adj0 = dv->adj0; wa.upper_off = dv->upper_off; wa.upper_adj = dv->upper_adj;
    wa.ep = dv->ep; wa.max_level = dv->max_level;
    wa.efp = P.efp; wa.efcap = (int)align_up(P.efp, 32);
    wa.R = P.R; wa.refine = P.refine ? 1 : 0;
    wa.beam = P.beam;
    wa.tcap = P.tcap;
    wa.hash_log = P.hash_log;
    wa.spill_log = P.spill_log;
    wa.spill = sc.spill;
    wa.status = sc.status;
    wa.counter = sc.counter;
    wa.stats_out = dstats;
    wa.yq_in = sc.yq;
    if (P.refine) {
        wa.yq_out = sc.yq;
        wa.short_out = sc.shortlist;
    } else {
        wa.ids_out = dids;
        wa.dists_out = ddists;
    }
    std::vector<int> off, len;
    splits(dv->d, dv->M1, off, len);
    for (int j = 0; j < dv->M1; j++) { wa.s1.off[j] = (uint16_t)off[j]; wa.s1.len[j] = (uint8_t)len[j]; }
    if (P.full) {
        wa.C2 = dv->C2;
        wa.C2h = static_cast<const __half *>(dv->C2h);
        wa.codes2b = dv->codes2b;
        wa.M2P = dv->M2P;
        std::vector<int> o2, l2;
        splits(dv->d, dv->M2, o2, l2);
        for (int j = 0; j < dv->M2; j++) for (int t = o2[j]; t < o2[j] + l2[j]; t++) wa.sub2[t] = (uint8_t)j;
    }
    if (cudaMemsetAsync(sc.status, 0, sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(sc.counter, 0, sizeof(unsigned long long), st) != cudaSuccess) {
        set_error("status reset failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    if (profile) {
        for (auto &e : dv->ev)
            if (!e) cudaEventCreate(&e);
        cudaEventRecord(dv->ev[0], st);
    }
    if (!rotated) rotate_kernel<<<std::max(P.qgrid, 1), ROT_THREADS, P.qsm, st>>>(dq, dq8, nq, dv->d, dv->Rt, sc.yq);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        set_error("rotation kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    ce = P.half ? run_any<__half>(P.variant, dv->M1, P.full, wa, P.smem, P.wpc, P.grid, st)
                : run_any<float>(P.variant, dv->M1, P.full, wa, P.smem, P.wpc, P.grid, st);
    if (profile) cudaEventRecord(dv->ev[1], st);
    if (ce != cudaSuccess) {
        set_error("walk kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    if (P.refine) {
        RefineArgs ra{};
        ra.yq = sc.yq; ra.shortlist = sc.shortlist; ra.nq = nq; ra.R = P.R; ra.k = P.k; ra.d = dv->d;
        ra.M1 = dv->M1; ra.M2P = dv->M2P; ra.C1 = dv->C1; ra.C2 = dv->C2; ra.B = dv->B;
        ra.codes1 = dv->codes1; ra.codes2b = dv->codes2b; ra.adj0 = dv->adj0;
        ra.ids_out = dids; ra.dists_out = ddists;
        std::vector<int> o2, l2;
        splits(dv->d, dv->M2, o2, l2);
        for (int j = 0; j < dv->M1; j++) for (int t = off[j]; t < off[j] + len[j]; t++) ra.sub1[t] = (uint8_t)j;
        for (int j = 0; j < dv->M2; j++) for (int t = o2[j]; t < o2[j] + l2[j]; t++) ra.sub2[t] = (uint8_t)j;
        std::vector<int> ob, lb;
        splits(dv->d, dv->bM, ob, lb);
        for (int m = 0; m < dv->bM; m++) for (int t = ob[m]; t < ob[m] + lb[m]; t++) ra.subb[t] = (uint8_t)m;
        ra.BM = dv->bM; ra.BK = dv->bK;
        auto kern = refine_kernel_for(P.rboth, dv->d, dv->bM > 1);
        kern<<<P.rgrid, P.rw * 32, P.rsm, st>>>(ra);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            set_error("refine kernel launch failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
    }
    if (profile) {
        cudaEventRecord(dv->ev[2], st);
        dv->ev_valid = true;
        dv->has_refine = P.refine;
    }
    return LC_OK;
}

lc_status search(lc_index *ix, const void *q, int qtype, int64_t nq, const lc_search_params *sp,
                 const int32_t *efq, int32_t *ids, float *dists, int32_t *stats, void *stream_)
{
    cudaStream_t st = (cudaStream_t)stream_;
    const int k = sp->k;
    // pointer kinds: all device or all host
    auto kind = [](const void *p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
    };
    int kq = kind(q), ki = kind(ids), kd = kind(dists), ks = stats ? kind(stats) : kq;
    int ke = efq ? kind(efq) : kq;
    if (kq != ki || kq != kd || kq != ks || kq != ke) {
        set_error("query, efSearch and output pointers must all be host or all be device memory");
        return LC_ERR_ARG;
    }
    const bool dev_ptrs = kq == 1;
    const bool u8 = qtype == LC_QUERY_U8;
    if (efq && !dev_ptrs) {
        for (int64_t i = 0; i < nq; i++)
            if (efq[i] < 1 || efq[i] > sp->ef) {
                set_error("efSearch of query %lld is %d, outside 1..%d", (long long)i, efq[i], sp->ef);
                return LC_ERR_ARG;
            }
    }
    lc_status rs = upload(ix);
    if (rs != LC_OK) return rs;
    DeviceIndex *dv = ix->dev;
    SearchPlan P;
    rs = plan_search(dv, std::max<int64_t>(nq, 1), sp, &P);
    if (rs != LC_OK) return rs;
    if (nq == 0) return LC_OK;
    const void *dq = q;
    const int32_t *defq = efq;
    int32_t *dids = ids, *dstats = stats;
    float *ddists = dists;
    if (!dev_ptrs) {
        if (!grow(dv->q_st, dv->q_cap, (size_t)nq * dv->d)) {
            set_error("cudaMalloc failed for query staging");
            return LC_ERR_OOM;
        }
        size_t need = (size_t)nq * std::max(k, 3);
        if (dv->out_cap < need || !dv->ids_st || !dv->d_st || !dv->s_st) {
            cfree(dv->ids_st); cfree(dv->d_st); cfree(dv->s_st);
            dv->ids_st = nullptr; dv->d_st = nullptr; dv->s_st = nullptr; dv->out_cap = 0;
            if (cudaMalloc(&dv->ids_st, need * 4) != cudaSuccess || cudaMalloc(&dv->d_st, need * 4) != cudaSuccess ||
                cudaMalloc(&dv->s_st, need * 4) != cudaSuccess) {
                set_error("cudaMalloc failed for search staging");
                return LC_ERR_OOM;
            }
            dv->out_cap = need;
        }
        if (efq && !grow(dv->ef_st, dv->ef_cap, (size_t)nq)) {
            set_error("cudaMalloc failed for efSearch staging");
            return LC_ERR_OOM;
        }
        if (cudaMemcpyAsync(dv->q_st, q, (u8 ? 1 : sizeof(float)) * nq * dv->d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            (efq && cudaMemcpyAsync(dv->ef_st, efq, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
            set_error("query upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            return LC_ERR_CUDA;
        }
        dq = dv->q_st;
        if (efq) defq = dv->ef_st;
        dids = dv->ids_st;
        ddists = dv->d_st;
        dstats = dv->s_st;
    }
    if (dv->n == 0) {
        // empty index: every result is padding
        std::vector<int32_t> hi((size_t)nq * k, -1);
        std::vector<float> hd((size_t)nq * k, INFINITY);
        std::vector<int32_t> hs((size_t)nq * 3, 0);
        cudaMemcpyKind kk = dev_ptrs ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        cudaMemcpy(ids, hi.data(), hi.size() * 4, kk);
        cudaMemcpy(dists, hd.data(), hd.size() * 4, kk);
        if (stats) cudaMemcpy(stats, hs.data(), hs.size() * 4, kk);
        return LC_OK;
    }
    if (!grow(dv->spill, dv->spill_cap, P.spill_elems) || !grow(dv->yq, dv->yq_cap, P.yq_elems) ||
        (P.refine && !grow(dv->shortlist, dv->sl_cap, P.sl_elems))) {
        set_error("cudaMalloc failed for search scratch");
        return LC_ERR_OOM;
    }
    SearchScratch sc;
    sc.yq = dv->yq;
    sc.shortlist = dv->shortlist;
    sc.spill = dv->spill;
    sc.status = dv->status;
    sc.counter = dv->counter;
    rs = run_search(dv, P, u8 ? nullptr : static_cast<const float *>(dq), nq, dids, ddists, dstats, sc, st,
                    dv->profile, u8 ? static_cast<const uint8_t *>(dq) : nullptr, defq);
    if (rs != LC_OK) return rs;
    if (!dev_ptrs) {
        cudaMemcpyAsync(ids, dids, sizeof(int32_t) * nq * k, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(dists, ddists, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st);
        if (stats) cudaMemcpyAsync(stats, dstats, sizeof(int32_t) * nq * 3, cudaMemcpyDeviceToHost, st);
        int32_t status = 0;
        cudaMemcpyAsync(&status, dv->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            set_error("search failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
        if (status) {
            set_error("a query's visited set overflowed its table (efSearch too large)");
            return LC_ERR_CAPACITY;
        }
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------------------
// Walk without allocation (lc_search_walk_noalloc).  Some callers cannot let the library call
// cudaMalloc while they serve: it may synchronise the whole device and take unbounded time,
// which a latency-bound request loop cannot afford, and an application that owns the device
// memory through its own pool or a fixed budget cannot have memory taken behind its back.
// This entry point runs the same walk kernel as lc_search, but its scratch (the query
// counter, the status word and the per-warp spill tables of the visited sets) lives in the
// file-scope array below, which every GPU that loads this library holds until exit.
constexpr int NOALLOC_SPILL_LOG = 12;                  // 4096 ids per query in flight
constexpr size_t NOALLOC_SLOTS = 2048;                 // queries in flight at most
constexpr size_t NOALLOC_HEADER = 256;                 // counter (8 B) and status (4 B)
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + NOALLOC_SLOTS * ((size_t)1 << NOALLOC_SPILL_LOG) * 4;
constexpr int NOALLOC_MAX_EF = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once per device.
static lc_status noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device %d is beyond the %d devices the no-allocation path tracks", dev, NOALLOC_MAX_DEVICES);
        return LC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
            return LC_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return LC_OK;
}

lc_status search_walk_noalloc(lc_index *ix, const float *q, int64_t nq, int k, int ef, int32_t *ids,
                              float *dists, int32_t *stats, void *stream_)
{
    cudaStream_t st = (cudaStream_t)stream_;
    const int efp = std::max(ef, k);
    if (efp > NOALLOC_MAX_EF) {
        set_error("max(ef, k) = %d exceeds %d, the widest walk the no-allocation scratch supports", efp,
                  NOALLOC_MAX_EF);
        return LC_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    DeviceIndex *dv = ix->dev;
    if (!dv || ix->dev_dirty || dv->device != dev) {
        set_error("index is not resident on device %d: run lc_search (which uploads it) first", dev);
        return LC_ERR_STATE;
    }
    auto on_device = [](const void *p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    };
    if (nq > 0 && (!on_device(q) || !on_device(ids) || !on_device(dists) || (stats && !on_device(stats)))) {
        set_error("the no-allocation walk takes device pointers only");
        return LC_ERR_ARG;
    }
    if (nq == 0) return LC_OK;
    if (dv->n == 0) {
        set_error("the no-allocation walk needs a non-empty index");
        return LC_ERR_STATE;
    }
    unsigned char *scratch = nullptr;
    lc_status s = noalloc_scratch(dev, &scratch);
    if (s != LC_OK) return s;

    WalkArgs wa{};
    wa.Q = q; wa.nq = nq; wa.d = dv->d;
    wa.Rt = dv->Rt; wa.C1 = dv->C1w; wa.codes1 = dv->codes1;
    wa.adj0 = dv->adj0; wa.upper_off = dv->upper_off; wa.upper_adj = dv->upper_adj;
    wa.ep = dv->ep; wa.max_level = dv->max_level;
    wa.efp = efp; wa.efcap = (int)align_up(efp, 32); wa.k = k;
    wa.R = k; wa.refine = 0;
    wa.beam = 1;
    wa.hash_log = std::min(12, std::max(10, ilog2_ceil((int64_t)efp * 32)));
    wa.spill_log = NOALLOC_SPILL_LOG;
    wa.ids_out = ids; wa.dists_out = dists; wa.stats_out = stats;
    wa.counter = reinterpret_cast<unsigned long long *>(scratch);
    wa.status = reinterpret_cast<int32_t *>(scratch + 8);
    wa.spill = reinterpret_cast<int32_t *>(scratch + NOALLOC_HEADER);
    std::vector<int> off, len;
    splits(dv->d, dv->M1, off, len);
    for (int j = 0; j < dv->M1; j++) { wa.s1.off[j] = (uint16_t)off[j]; wa.s1.len[j] = (uint8_t)len[j]; }
    const size_t per_warp = walk_smem(dv->M1, dv->d, wa.efcap, wa.hash_log, wa.beam, true).total;
    const int variant = (dv->M1 == 16 && dv->d == 96) ? 1 : (dv->M1 == 32 && dv->d == 96) ? 2
                      : (dv->M1 == 64 && dv->d == 128) ? 3 : 0;
    int grid = 0, wpc = 1;
    size_t smem = 0;
    cudaError_t ce;
    ce = launch_any<float>(variant, dv->M1, false, wa, per_warp, dv->num_sms, 0, &wpc, &grid, &smem);
    if (ce != cudaSuccess) {
        set_error("walk kernel configuration failed: %s", cudaGetErrorString(ce));
        return ce == cudaErrorInvalidConfiguration ? LC_ERR_CAPACITY : LC_ERR_CUDA;
    }
    // every warp in flight owns one spill table of the array
    grid = (int)std::min<int64_t>(grid, (int64_t)(NOALLOC_SLOTS / wpc));
    // the array keeps the previous call's contents: the counter and status start at zero
    // (spill tables are cleared by the kernel before a query uses one)
    if (cudaMemsetAsync(scratch, 0, 16, st) != cudaSuccess) {
        set_error("reset of the no-allocation scratch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    ce = run_any<float>(variant, dv->M1, false, wa, smem, wpc, grid, st);
    if (ce != cudaSuccess) {
        set_error("walk kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------------------
// Top-k merge of per-shard results (sharded search: every query searches every shard, then
// the shards' k best are merged by (distance, global id)).  One warp per query: the S*k keys
// (shard-local ids shifted by the shard's id offset) are sorted in shared memory by a bitonic
// network and the k smallest are written.
constexpr int MERGE_MAX = 2048;   // S * k per query
constexpr int MERGE_WARPS = 4;
constexpr int MERGE_MAX_SHARDS = 64;

struct ShardOffsets {
    int64_t v[MERGE_MAX_SHARDS];
};

__global__ void __launch_bounds__(MERGE_WARPS * 32) merge_kernel(const int32_t *ids, const float *dists,
                                                                 int S, int64_t nq, int k,
                                                                 const ShardOffsets offsets, int32_t *ids_out,
                                                                 float *dists_out, int P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem_raw) + (size_t)warp * P;
    const int64_t gwarp = (int64_t)blockIdx.x * MERGE_WARPS + warp;
    const int64_t nwarps = (int64_t)gridDim.x * MERGE_WARPS;
    for (int64_t q = gwarp; q < nq; q += nwarps) {
        for (int i = lane; i < P; i += 32) {
            uint64_t key = ~0ull;
            if (i < S * k) {
                const int s = i / k, j = i % k;
                const int64_t src = ((int64_t)s * nq + q) * k + j;
                const int32_t id = ids[src];
                if (id >= 0) key = make_key(dists[src], (int32_t)(id + offsets.v[s]));
            }
            keys[i] = key;
        }
        __syncwarp();
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int p = i ^ j;
                    if (p > i) {
                        const uint64_t x = keys[i], y = keys[p];
                        const bool up = (i & kk) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[p] = x; }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < k; i += 32) {
            const uint64_t key = keys[i];
            const bool ok = key != ~0ull;
            ids_out[q * k + i] = ok ? key_id(key) : -1;
            dists_out[q * k + i] = ok ? key_dist(key) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

lc_status merge_topk(const int32_t *ids, const float *dists, int S, int64_t nq, int k, const int64_t *offsets,
                     int32_t *ids_out, float *dists_out, void *stream_)
{
    cudaStream_t st = (cudaStream_t)stream_;
    if (nq == 0) return LC_OK;
    int P = 32;
    while (P < S * k) P <<= 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ShardOffsets off{};
    for (int i = 0; i < S; i++) off.v[i] = offsets[i];
    const size_t smem = (size_t)P * 8 * MERGE_WARPS;
    cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_SMEM_PER_BLOCK);
    const int64_t need = (nq + MERGE_WARPS - 1) / MERGE_WARPS;
    const int grid = (int)std::min<int64_t>(need, (int64_t)sms * 8);
    merge_kernel<<<grid, MERGE_WARPS * 32, smem, st>>>(ids, dists, S, nq, k, off, ids_out, dists_out, P);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        set_error("merge kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    return LC_OK;
}


// ------------------------------------------------------------------------------------------
// Captured searches.  A plan fixes the search parameters and a largest batch, owns its device
// buffers (queries, per-query efSearch, outputs and the walk's scratch) and records the whole
// search -- counter and status resets, walk, re-rank -- into one CUDA graph, so that a call
// is a single graph launch with no planning, allocation or attribute calls on the host.  A
// batch smaller than the largest updates the batch size in the two kernel nodes of the
// executable graph (launches already queued keep the size they were launched with).
}  // namespace lc

struct lc_plan {
    lc_index *ix = nullptr;
    uint64_t gen = 0;
    int device = -1;
    lc::SearchPlan P;
    int qtype = LC_QUERY_F32;
    bool per_query_ef = false;
    int64_t nq_max = 0, nq_cur = 0;
    void *q = nullptr;
    int32_t *ef = nullptr, *ids = nullptr, *stats = nullptr;
    float *dists = nullptr;
    lc::SearchScratch sc;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t walk_node = nullptr, refine_node = nullptr;
    cudaKernelNodeParams walk_kp{}, refine_kp{};
    lc::WalkArgs wa{};
    lc::RefineArgs ra{};
};

namespace lc {

void plan_free(lc_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    cfree(pl->q); cfree(pl->ef); cfree(pl->ids); cfree(pl->dists); cfree(pl->stats);
    cfree(pl->sc.yq); cfree(pl->sc.shortlist); cfree(pl->sc.spill); cfree(pl->sc.status); cfree(pl->sc.counter);
    delete pl;
}

lc_status plan_create(lc_index *ix, int64_t nq_max, const lc_search_params *sp, int qtype, int per_query_ef,
                      lc_plan **out)
{
    lc_status rs = upload(ix);
    if (rs != LC_OK) return rs;
    DeviceIndex *dv = ix->dev;
    if (dv->n == 0) {
        set_error("plans need a non-empty index");
        return LC_ERR_STATE;
    }
    lc_plan *pl = new lc_plan();
    pl->ix = ix;
    pl->gen = dv->gen;
    pl->device = dv->device;
    pl->qtype = qtype;
    pl->per_query_ef = per_query_ef != 0;
    pl->nq_max = nq_max;
    pl->nq_cur = nq_max;
    rs = plan_search(dv, nq_max, sp, &pl->P);
    if (rs != LC_OK) { plan_free(pl); return rs; }
    const SearchPlan &P = pl->P;
    const int d = dv->d, k = sp->k;
    auto alloc = [&](auto *&p, size_t bytes) { return cudaMalloc(&p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
    bool ok = alloc(pl->q, (size_t)nq_max * d * (qtype == LC_QUERY_U8 ? 1 : 4)) &&
              (!pl->per_query_ef || alloc(pl->ef, (size_t)nq_max * 4)) &&
              alloc(pl->ids, (size_t)nq_max * k * 4) && alloc(pl->dists, (size_t)nq_max * k * 4) &&
              alloc(pl->stats, (size_t)nq_max * 12) && alloc(pl->sc.spill, P.spill_elems * 4) &&
              alloc(pl->sc.status, 4) && alloc(pl->sc.counter, 8) &&
              alloc(pl->sc.yq, P.yq_elems * 4) && (!P.refine || alloc(pl->sc.shortlist, P.sl_elems * 4));
    if (!ok) {
        plan_free(pl);
        set_error("cudaMalloc failed for the plan's buffers");
        return LC_ERR_OOM;
    }
    if (pl->per_query_ef) {
        // every query starts at the plan's efSearch until the caller writes its own
        std::vector<int32_t> e((size_t)nq_max, sp->ef);
        cudaMemcpy(pl->ef, e.data(), e.size() * 4, cudaMemcpyHostToDevice);
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        plan_free(pl);
        set_error("stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        const bool u8 = qtype == LC_QUERY_U8;
        rs = run_search(dv, P, u8 ? nullptr : static_cast<const float *>(pl->q), nq_max, pl->ids, pl->dists,
                        pl->stats, pl->sc, st, false, u8 ? static_cast<const uint8_t *>(pl->q) : nullptr,
                        pl->per_query_ef ? pl->ef : nullptr);
        cudaError_t ce2 = cudaStreamEndCapture(st, &pl->graph);
        if (rs == LC_OK && ce2 != cudaSuccess) ce = ce2;
    }
    cudaStreamDestroy(st);
    if (ce != cudaSuccess || rs != LC_OK) {
        if (rs == LC_OK) set_error("capture of the search failed: %s", cudaGetErrorString(ce));
        plan_free(pl);
        return rs == LC_OK ? LC_ERR_CUDA : rs;
    }
    // find the two kernel nodes whose batch size a smaller call updates
    const void *wf = P.half ? walk_fn<__half>(P.variant, dv->M1, P.full) : walk_fn<float>(P.variant, dv->M1, P.full);
    const void *rf = P.refine ? (const void *)refine_kernel_for(P.rboth, d, dv->bM > 1) : nullptr;
    size_t nn = 0;
    cudaGraphGetNodes(pl->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(pl->graph, nodes.data(), &nn);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        if (kp.func == wf) {
            pl->walk_node = nd;
            pl->walk_kp = kp;
            pl->wa = *static_cast<const WalkArgs *>(kp.kernelParams[0]);
        } else if (rf && kp.func == rf) {
            pl->refine_node = nd;
            pl->refine_kp = kp;
            pl->ra = *static_cast<const RefineArgs *>(kp.kernelParams[0]);
        }
    }
    if (!pl->walk_node || (P.refine && !pl->refine_node)) {
        plan_free(pl);
        set_error("captured search graph lacks its kernels");
        return LC_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (ce != cudaSuccess) {
        plan_free(pl);
        set_error("graph instantiation failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    *out = pl;
    return LC_OK;
}

lc_status plan_buffers(const lc_plan *pl, void **q, int32_t **ef, int32_t **ids, float **dists, int32_t **stats)
{
    if (q) *q = pl->q;
    if (ef) *ef = pl->ef;
    if (ids) *ids = pl->ids;
    if (dists) *dists = pl->dists;
    if (stats) *stats = pl->stats;
    return LC_OK;
}

lc_status plan_run(lc_plan *pl, int64_t nq, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (nq < 0 || nq > pl->nq_max) {
        set_error("nq = %lld outside 0..%lld", (long long)nq, (long long)pl->nq_max);
        return LC_ERR_ARG;
    }
    lc_index *ix = pl->ix;
    if (ix->dev_dirty || !ix->dev || ix->dev->gen != pl->gen) {
        set_error("the index changed since the plan was made; make a new plan");
        return LC_ERR_STATE;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != pl->device) {
        set_error("plan made on device %d, current device is %d", pl->device, dev);
        return LC_ERR_STATE;
    }
    if (nq == 0) return LC_OK;
    if (nq != pl->nq_cur) {
        pl->wa.nq = nq;
        void *wp[1] = {&pl->wa};
        cudaKernelNodeParams kp = pl->walk_kp;
        kp.kernelParams = wp;
        cudaError_t ce = cudaGraphExecKernelNodeSetParams(pl->exec, pl->walk_node, &kp);
        if (ce == cudaSuccess && pl->refine_node) {
            pl->ra.nq = nq;
            void *rp[1] = {&pl->ra};
            cudaKernelNodeParams kr = pl->refine_kp;
            kr.kernelParams = rp;
            ce = cudaGraphExecKernelNodeSetParams(pl->exec, pl->refine_node, &kr);
        }
        if (ce != cudaSuccess) {
            set_error("updating the plan's batch size failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
        pl->nq_cur = nq;
    }
    cudaError_t ce = cudaGraphLaunch(pl->exec, st);
    if (ce != cudaSuccess) {
        set_error("graph launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------------------
// GPU-assisted build.  lc_add inserts by batches, each searching the graph as it stood at the
// batch start (Section 5.1); the level-0 insertion searches of a batch are independent, so
// they run as one launch of the walk on the device copy of the index, with the exact-to-
// decoded distance of the full-decode walk (FP32).  The host keeps neighbour selection,
// linking and the nodes of higher level, and re-sends the rows a batch changed.

__global__ void scatter_rows_kernel(int32_t *dst, const int64_t *idx, const int32_t *rows, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * DEG; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i / DEG] * DEG + (i % DEG)] = rows[i];
}

// Neighbour selection of the GPU-assisted build: HNSW's shrinking heuristic on each member's
// candidate list (sorted by distance to the member): a candidate is kept unless it is closer to
// an already kept neighbour than to the member, up to DEG kept.  One warp per member; lane u
// tests the candidate against the u-th kept neighbour.  The decoded-to-decoded distance
// reproduces the host build's float arithmetic (eight partial sums over coordinate groups,
// then a fixed tree; no multiply-add contraction), so the choices are the host's.
struct SelectArgs {
    const int32_t *cand_ids;          // [m][efc], -1 padded
    const float *cand_d;              // [m][efc]
    int32_t *sel;                     // [m][DEG + 1]: kept ids, then their count
    int64_t m;
    int efc, d, M1, M2P;
    const float *C1, *C2;
    const uint8_t *codes1, *codes2b;
    uint8_t sub1[256], sub2[256];
};

__device__ __forceinline__ float decoded_at(const SelectArgs &a, int32_t v, int t)
{
    return __fadd_rn(__ldg(a.C1 + (int)__ldg(a.codes1 + (int64_t)v * a.M1 + a.sub1[t]) * a.d + t),
                     __ldg(a.C2 + (int)__ldg(a.codes2b + (int64_t)v * a.M2P + a.sub2[t]) * a.d + t));
}

__device__ float decoded_l2(const SelectArgs &a, int32_t p, int32_t q)
{
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int t = 0;
    for (; t + 8 <= a.d; t += 8) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const float x = __fsub_rn(decoded_at(a, p, t + u), decoded_at(a, q, t + u));
            s[u] = __fadd_rn(s[u], __fmul_rn(x, x));
        }
    }
    for (; t < a.d; t++) {
        const float x = __fsub_rn(decoded_at(a, p, t), decoded_at(a, q, t));
        s[0] = __fadd_rn(s[0], __fmul_rn(x, x));
    }
    return __fadd_rn(__fadd_rn(__fadd_rn(s[0], s[1]), __fadd_rn(s[2], s[3])),
                     __fadd_rn(__fadd_rn(s[4], s[5]), __fadd_rn(s[6], s[7])));
}

__global__ void __launch_bounds__(256) select_kernel(const SelectArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t mi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (mi >= a.m) return;                               // whole warps leave together
    const int32_t *ci = a.cand_ids + mi * a.efc;
    const float *cd = a.cand_d + mi * a.efc;
    int kept = 0;
    int32_t kid = -1;                                    // lane u: the u-th kept neighbour
    for (int s = 0; s < a.efc && kept < DEG; s++) {
        const int32_t c = __ldg(ci + s);
        if (c < 0) break;
        const float dc = __ldg(cd + s);
        const bool closer = lane < kept && decoded_l2(a, c, kid) < dc;
        if (__ballot_sync(FULL, closer) == 0) {
            if (lane == kept) kid = c;
            kept++;
        }
    }
    int32_t *out = a.sel + mi * (DEG + 1);
    out[lane] = lane < kept ? kid : -1;
    if (lane == 0) out[DEG] = kept;
}

lc_status build_gpu_begin(lc_index *ix)
{
    ix->dev_dirty = true;                       // upload the index as it stands (codes of all nodes)
    return upload(ix);
}

lc_status build_gpu_search(lc_index *ix, const float *xr, int64_t m, int efc, int32_t ep, int max_level,
                           int32_t *ids, float *dists, int32_t *sel)
{
    DeviceIndex *dv = ix->dev;
    if (!dv || m <= 0) return LC_OK;
    lc_search_params sp;
    lc_default_search_params(&sp, efc, efc);
    sp.shortlist = -1;                          // the walk's own result list, sorted
    sp.walk_full = 1;
    SearchPlan P;
    lc_status rs = plan_search(dv, m, &sp, &P);
    if (rs != LC_OK) return rs;
    if (!grow(dv->b_yq, dv->b_yq_cap, (size_t)m * dv->d) || !grow(dv->b_ids, dv->b_ids_cap, (size_t)m * efc) ||
        !grow(dv->b_d, dv->b_d_cap, (size_t)m * efc) || !grow(dv->spill, dv->spill_cap, P.spill_elems)) {
        set_error("cudaMalloc failed for the build's search buffers");
        return LC_ERR_OOM;
    }
    if (cudaMemcpy(dv->b_yq, xr, sizeof(float) * m * dv->d, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("build batch upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    dv->ep = ep;
    dv->max_level = max_level < 0 ? 0 : max_level;
    SearchScratch sc;
    sc.yq = dv->b_yq;
    sc.spill = dv->spill;
    sc.status = dv->status;
    sc.counter = dv->counter;
    rs = run_search(dv, P, nullptr, m, dv->b_ids, dv->b_d, nullptr, sc, 0, false, nullptr, nullptr, true);
    if (rs != LC_OK) return rs;
    int32_t status = 0;
    bool ok;
    if (sel) {
        // neighbour selection on the device; only the selections come back
        if (!grow(dv->b_sel, dv->b_sel_cap, (size_t)m * (DEG + 1))) {
            set_error("cudaMalloc failed for the build's selections");
            return LC_ERR_OOM;
        }
        SelectArgs sa{};
        sa.cand_ids = dv->b_ids; sa.cand_d = dv->b_d; sa.sel = dv->b_sel; sa.m = m; sa.efc = efc;
        sa.d = dv->d; sa.M1 = dv->M1; sa.M2P = dv->M2P; sa.C1 = dv->C1; sa.C2 = dv->C2;
        sa.codes1 = dv->codes1; sa.codes2b = dv->codes2b;
        std::vector<int> o, l;
        splits(dv->d, dv->M1, o, l);
        for (int j = 0; j < dv->M1; j++) for (int t = o[j]; t < o[j] + l[j]; t++) sa.sub1[t] = (uint8_t)j;
        splits(dv->d, dv->M2, o, l);
        for (int j = 0; j < dv->M2; j++) for (int t = o[j]; t < o[j] + l[j]; t++) sa.sub2[t] = (uint8_t)j;
        select_kernel<<<(unsigned)((m * 32 + 255) / 256), 256>>>(sa);
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemcpy(sel, dv->b_sel, sizeof(int32_t) * m * (DEG + 1), cudaMemcpyDeviceToHost) == cudaSuccess;
    } else {
        ok = cudaMemcpy(ids, dv->b_ids, sizeof(int32_t) * m * efc, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(dists, dv->b_d, sizeof(float) * m * efc, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (!ok || cudaMemcpy(&status, dv->status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("build search failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    if (status) {
        set_error("an insertion search overflowed its visited table");
        return LC_ERR_CAPACITY;
    }
    return LC_OK;
}

static lc_status scatter_rows(DeviceIndex *dv, int32_t *dst, const int32_t *src_rows, const int64_t *idx, int64_t n)
{
    if (n <= 0) return LC_OK;
    std::vector<int32_t> rows((size_t)n * DEG);
    for (int64_t r = 0; r < n; r++) std::memcpy(rows.data() + r * DEG, src_rows + idx[r] * DEG, DEG * 4);
    if (!grow(dv->b_rows, dv->b_rows_cap, rows.size()) || !grow(dv->b_idx, dv->b_idx_cap, (size_t)n)) {
        set_error("cudaMalloc failed for the build's row updates");
        return LC_ERR_OOM;
    }
    if (cudaMemcpy(dv->b_rows, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dv->b_idx, idx, (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("row update upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    const int grid = (int)std::min<int64_t>((n * DEG + 255) / 256, (int64_t)dv->num_sms * 8);
    scatter_rows_kernel<<<grid, 256>>>(dst, dv->b_idx, dv->b_rows, n);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("row update launch failed");
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

lc_status build_gpu_rows(lc_index *ix, const int32_t *nodes0, int64_t n0, const int64_t *rows_up, int64_t nu)
{
    DeviceIndex *dv = ix->dev;
    if (!dv) return LC_OK;
    std::vector<int64_t> i0(nodes0, nodes0 + n0);
    lc_status rs = scatter_rows(dv, dv->adj0, ix->adj0.data(), i0.data(), n0);
    if (rs != LC_OK) return rs;
    return scatter_rows(dv, dv->upper_adj, ix->upper_adj.data(), rows_up, nu);
}

// Codeword assignment on the device (Section 4.3): one thread per vector computes the normal
// equations of each regression block over its coordinates in the host build's order (sums
// over t ascending, double, multiply and add rounded separately as the host compiles them) and
// takes the argmin over the block's codewords (first minimum), so the choice is the host's.
struct AssignArgs {
    const float *xr;                  // rotated vectors of this chunk [n][d]
    int64_t first, n;                 // global id of row 0, rows
    int d, M1, M2P, bM, bK;
    const float *C1, *C2, *B;         // [256][d], [256][d], [bM][bK][9]
    const uint8_t *codes1, *codes2b;
    const int32_t *adj0;
    uint8_t *beta_out;                // [n][bM]
    uint8_t sub1[256], sub2[256];     // level-1 / level-2 sub-space of each coordinate
    uint16_t boff[33];                // regression block m covers [boff[m], boff[m + 1])
};

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

__global__ void __launch_bounds__(128) assign_kernel(const AssignArgs a)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.n) return;
    const int64_t i = a.first + v;
    int32_t vid[9];
    vid[0] = (int32_t)i;
    for (int j = 1; j <= 8; j++) vid[j] = __ldg(a.adj0 + i * DEG + j - 1);
    const float *x = a.xr + v * a.d;
    for (int m = 0; m < a.bM; m++) {
        double A[45], b[9], xx = 0.0;
        for (int u = 0; u < 45; u++) A[u] = 0.0;
        for (int u = 0; u < 9; u++) b[u] = 0.0;
        for (int t = a.boff[m]; t < a.boff[m + 1]; t++) {
            // q(v) at coordinate t: level-1 plus level-2 centroid, added in FP32 as the host decodes
            float g[9];
#pragma unroll
            for (int j = 0; j < 9; j++)
                g[j] = vid[j] < 0 ? 0.f
                       : __ldg(a.C1 + (int)__ldg(a.codes1 + (int64_t)vid[j] * a.M1 + a.sub1[t]) * a.d + t) +
                             __ldg(a.C2 + (int)__ldg(a.codes2b + (int64_t)vid[j] * a.M2P + a.sub2[t]) * a.d + t);
            const double xt = (double)__ldg(x + t);
            int u = 0;
#pragma unroll
            for (int p = 0; p < 9; p++) {
                if (vid[p] >= 0) b[p] = dadd(b[p], dmul((double)g[p], xt));
#pragma unroll
                for (int c = p; c < 9; c++, u++)
                    if (vid[p] >= 0 && vid[c] >= 0) A[u] = dadd(A[u], dmul((double)g[p], (double)g[c]));
            }
            xx = dadd(xx, dmul(xt, xt));
        }
        int best = 0;
        if (a.bK > 1) {
            double bl = __longlong_as_double(0x7ff0000000000000ll);        // +inf
            for (int cw = 0; cw < a.bK; cw++) {
                const float *bw = a.B + ((int64_t)m * a.bK + cw) * 9;
                double be[9];
#pragma unroll
                for (int p = 0; p < 9; p++) be[p] = (double)__ldg(bw + p);
                // ||x - beta^T G||^2 = ||x||^2 - 2 beta.b + beta^T A beta, in the host's order
                double sl = xx;
                int u = 0;
#pragma unroll
                for (int p = 0; p < 9; p++) {
                    sl = dsub(sl, dmul(dmul(2.0, be[p]), b[p]));
                    sl = dadd(sl, dmul(dmul(be[p], be[p]), A[u]));
                    u++;
#pragma unroll
                    for (int c = p + 1; c < 9; c++, u++) sl = dadd(sl, dmul(dmul(dmul(2.0, be[p]), be[c]), A[u]));
                }
                if (sl < bl) { bl = sl; best = cw; }
            }
        }
        a.beta_out[v * a.bM + m] = (uint8_t)best;
    }
}

lc_status build_gpu_assign(lc_index *ix, const float *xr, int64_t first, int64_t n)
{
    lc_status rs = LC_OK;
    if (!ix->dev) {
        rs = upload(ix);
        if (rs != LC_OK) return rs;
    }
    DeviceIndex *dv = ix->dev;
    const int d = ix->p.d, bM = ix->p.beta_M, bK = ix->p.beta_K;
    if (!dupload(dv->B, ix->B)) {                   // trained after the graph
        set_error("upload of the regression codebook failed");
        return LC_ERR_OOM;
    }
    AssignArgs aa{};
    aa.d = d; aa.M1 = ix->p.M1; aa.M2P = dv->M2P; aa.bM = bM; aa.bK = bK;
    aa.C1 = dv->C1; aa.C2 = dv->C2; aa.B = dv->B;
    aa.codes1 = dv->codes1; aa.codes2b = dv->codes2b; aa.adj0 = dv->adj0;
    std::vector<int> o, l;
    splits(d, ix->p.M1, o, l);
    for (int j = 0; j < ix->p.M1; j++) for (int t = o[j]; t < o[j] + l[j]; t++) aa.sub1[t] = (uint8_t)j;
    splits(d, ix->p.M2, o, l);
    for (int j = 0; j < ix->p.M2; j++) for (int t = o[j]; t < o[j] + l[j]; t++) aa.sub2[t] = (uint8_t)j;
    splits(d, bM, o, l);
    for (int m = 0; m < bM; m++) aa.boff[m] = (uint16_t)o[m];
    aa.boff[bM] = (uint16_t)d;
    const int64_t CH = 1 << 20;                      // vectors per chunk
    uint8_t *dbeta = nullptr;
    size_t xcap = 0;
    float *dx = nullptr;
    if (cudaMalloc(&dbeta, (size_t)std::min(n, CH) * bM + 16) != cudaSuccess) {
        set_error("cudaMalloc failed for codeword assignment");
        return LC_ERR_OOM;
    }
    for (int64_t c0 = 0; c0 < n && rs == LC_OK; c0 += CH) {
        const int64_t m = std::min(CH, n - c0);
        if (!grow(dx, xcap, (size_t)m * d) ||
            cudaMemcpy(dx, xr + c0 * d, sizeof(float) * m * d, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("upload for codeword assignment failed");
            rs = LC_ERR_CUDA;
            break;
        }
        aa.xr = dx; aa.first = first + c0; aa.n = m; aa.beta_out = dbeta;
        assign_kernel<<<(unsigned)((m + 127) / 128), 128>>>(aa);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(ix->beta.data() + (first + c0) * bM, dbeta, (size_t)m * bM, cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("codeword assignment on the device failed: %s", cudaGetErrorString(cudaGetLastError()));
            rs = LC_ERR_CUDA;
        }
    }
    cfree(dx);
    cfree(dbeta);
    ix->dev_dirty = true;
    return rs;
}

void build_gpu_end(lc_index *ix)
{
    DeviceIndex *dv = ix->dev;
    if (dv) {
        cudaDeviceSynchronize();
        cfree(dv->b_yq); cfree(dv->b_ids); cfree(dv->b_d); cfree(dv->b_rows); cfree(dv->b_idx); cfree(dv->b_sel);
        dv->b_yq = nullptr; dv->b_ids = nullptr; dv->b_d = nullptr; dv->b_rows = nullptr; dv->b_idx = nullptr;
        dv->b_sel = nullptr;
        dv->b_yq_cap = dv->b_ids_cap = dv->b_d_cap = dv->b_rows_cap = dv->b_idx_cap = dv->b_sel_cap = 0;
    }
    ix->dev_dirty = true;                       // codewords are assigned after the graph
}

lc_status profile_enable(lc_index *ix, int on)
{
    lc_status s = upload(ix);
    if (s != LC_OK) return s;
    ix->dev->profile = on != 0;
    ix->dev->ev_valid = false;
    return LC_OK;
}

lc_status profile_read(lc_index *ix, float *walk_ms, float *refine_ms)
{
    if (!ix->dev || !ix->dev->profile || !ix->dev->ev_valid) {
        set_error("no profiled search to read");
        return LC_ERR_STATE;
    }
    DeviceIndex *dv = ix->dev;
    if (cudaEventSynchronize(dv->ev[2]) != cudaSuccess) {
        set_error("event synchronisation failed");
        return LC_ERR_CUDA;
    }
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, dv->ev[0], dv->ev[1]);
    if (dv->has_refine) cudaEventElapsedTime(&b, dv->ev[1], dv->ev[2]);
    if (walk_ms) *walk_ms = a;
    if (refine_ms) *refine_ms = b;
    return LC_OK;
}

}  // namespace lc
