// GPU search path of Link and Code (Douze, Sablayrolles, Jegou, CVPR 2018), sm_103a: the
// host side of a search and the kernels other than the walk (which is in lc_walk.cuh).
//
// rotate_kernel  y' = R y for a batch of queries (OPQ rotation, Section 3.3 / 5.1).
// table_kernel   per-query ADC tables on the tensor cores (the LC_LUT_TABLE form, Section 4.1).
// order_kernel   queue order of an ordered search (decreasing distance to the level-0 entry).
// walk           lc_walk.cuh / lc_walk_f32.cu / lc_walk_f16.cu: upper-level descent and level-0
//                search (Section 2) scored by ADC on the level-1 code (Section 4.1).
// refine_kernel  (one warp per query) for each shortlisted x: G(x) = [q(x), q(g_1..g_8)]
//                decoded from both code levels, y^ = beta_b^T G(x) with b the vector's codeword
//                (per block with a product codebook; Section 4.2, 4.3), exact squared L2 to
//                y', and the final top-k by (distance, id).
// merge_kernel   top-k merge of per-shard results (sharded search).
// Host side      device copy of the index (upload), launch planning (plan_search), one search
//                (run_search / search), captured plans (lc_plan_*), the walk without
//                allocation, and kernel timing.  The GPU-assisted build is in lc_build_gpu.cu.
//
// Ordering everywhere is by (distance, id), smaller id first on equal distances.

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lc_walk.cuh"

namespace lc {


void device_free(DeviceIndex *dv)
{
    if (!dv) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (dv->device >= 0) cudaSetDevice(dv->device);
    cfree(dv->Rt); cfree(dv->C1); cfree(dv->C2); cfree(dv->B); cfree(dv->C1h); cfree(dv->C1w); cfree(dv->C2h);
    cfree(dv->codes1); cfree(dv->codes2b);
    cfree(dv->adj0); cfree(dv->upper_off); cfree(dv->upper_adj);
    cfree(dv->yq); cfree(dv->shortlist); cfree(dv->spill); cfree(dv->ord); cfree(dv->status); cfree(dv->counter);
    cfree(dv->tab);
    cfree(dv->b_yq); cfree(dv->b_ids); cfree(dv->b_d); cfree(dv->b_rows); cfree(dv->b_idx); cfree(dv->b_sel);
    link0_free(dv);
    cfree(dv->q_st); cfree(dv->ef_st); cfree(dv->ids_st); cfree(dv->d_st); cfree(dv->s_st);
    for (auto &e : dv->ev) if (e) cudaEventDestroy(e);
    if (cur >= 0) cudaSetDevice(cur);
    delete dv;
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

// ------------------------------------------------------------------------------------------
// Queue order of the ordered search: the queries sorted by decreasing distance to their
// level-0 entry node (a query whose upper-level descent stopped far from it tends to walk
// long at level 0, so those start first and the launch does not end on a few long walks).
// One block of ORDER_THREADS threads: a histogram of the distances over ORDER_BUCKETS buckets
// (the float's exponent and top 3 mantissa bits: distances are non-negative, so the bit
// pattern orders like the value), exclusive sums in decreasing bucket order, then a scatter.
// Within a bucket the order is whatever the atomics give; results do not depend on it.
constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_BUCKETS = 2 * ORDER_THREADS;     // each thread sums two buckets
constexpr int ORDER_MIN_ROUNDS = 2;                  // auto: queries >= 2 x warps in flight

__device__ __forceinline__ int order_bucket(float x)
{
    return (int)((__float_as_uint(x) & 0x7fffffffu) >> 20);          // 0 .. 2047
}

__global__ void __launch_bounds__(ORDER_THREADS) order_kernel(const float *key, int64_t n, int32_t *order)
{
    __shared__ uint32_t pos[ORDER_BUCKETS];
    __shared__ uint32_t wsum[ORDER_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int i = t; i < ORDER_BUCKETS; i += ORDER_THREADS) pos[i] = 0;
    __syncthreads();
    for (int64_t i = t; i < n; i += ORDER_THREADS) atomicAdd(&pos[order_bucket(__ldg(key + i))], 1u);
    __syncthreads();
    // thread t owns buckets b0 = 2047 - 2t and b0 - 1 (ranks 2t and 2t + 1 in decreasing order)
    const int b0 = ORDER_BUCKETS - 1 - 2 * t, b1 = b0 - 1;
    const uint32_t c0 = pos[b0], c1 = pos[b1];
    const uint32_t own = c0 + c1;
    uint32_t inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t v = wsum[lane];
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += u;
        }
        wsum[lane] = vi - v;                          // warps before this one
    }
    __syncthreads();
    const uint32_t ex = wsum[w] + inc - own;          // queries in buckets above b0
    pos[b0] = ex;                                     // only this thread reads or writes b0, b1
    pos[b1] = ex + c0;
    __syncthreads();
    for (int64_t i = t; i < n; i += ORDER_THREADS) {
        const uint32_t p = atomicAdd(&pos[order_bucket(__ldg(key + i))], 1u);
        order[p] = (int32_t)i;
    }
}

// Per-query ADC tables on the tensor cores (table_kernel, search form LC_LUT_TABLE), for the
// uniform split of 96 coordinates into 32 sub-spaces of 3: for query q, sub-space j and
// centroid c, T[q][c][j] = ||y'_j||^2 + ||C1_j[c]||^2 - 2 <y'_j, C1_j[c]> (Section 4.1's ADC
// table), with y' and C1 rounded to FP16 (C1 is the walk's FP16 codebook), the inner products
// taken by FP16 tensor-core products with FP32 accumulation (mma.sync m16n8k8: 16 centroids x
// 8 queries, the sub-space's 3 coordinates padded to the 8 of the instruction), the norms in
// FP32 from the same rounded values, the entry rounded to FP16.  One warp builds the tables of
// 8 queries: per block of 16 centroids a lane gathers its 4 (centroid, query) entries over the
// 32 sub-spaces and writes them as 64-byte rows, so each query's table is one contiguous
// 16 KB block [256][32] (the layout the table walk copies into shared memory).
constexpr int TAB_WARPS = 4;
constexpr int TAB_M1 = 32;

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(TAB_WARPS * 32) table_kernel(const float *yq, int64_t nq, const __half *C1h,
                                                               __half *T)
{
    constexpr int M1 = TAB_M1, D = 96;
    // the FP16 codebook in the walk's split layout: half2 [256][32] (coordinates 0, 1 of every
    // sub-space), then half [256][32] (coordinate 2)
    __shared__ __align__(16) __half cb[256 * M1 * 3];
    for (int i = threadIdx.x; i < 256 * M1 * 3 / 8; i += blockDim.x)
        reinterpret_cast<uint4 *>(cb)[i] = __ldg(reinterpret_cast<const uint4 *>(C1h) + i);
    __syncthreads();
    const __half2 *cb2 = reinterpret_cast<const __half2 *>(cb);
    const __half *cb1 = cb + 256 * M1 * 2;
    const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
    const int64_t q0 = ((int64_t)blockIdx.x * TAB_WARPS + (threadIdx.x >> 5)) * 8;
    if (q0 >= nq) return;
    // B fragments (8 queries: query g, coordinates 2tg, 2tg + 1 of each sub-space) and the
    // queries' sub-space norms, for all 32 sub-spaces
    const int64_t qb = min(q0 + g, nq - 1);
    uint32_t bf[M1];
    float yn[M1];
#pragma unroll
    for (int j = 0; j < M1; j++) {
        float y0 = 0.f, y1 = 0.f;
        if (tg == 0) { y0 = __ldg(yq + qb * D + 3 * j); y1 = __ldg(yq + qb * D + 3 * j + 1); }
        if (tg == 1) y0 = __ldg(yq + qb * D + 3 * j + 2);
        bf[j] = pack_half2(y0, y1);
        const __half2 h = *reinterpret_cast<const __half2 *>(&bf[j]);
        const float r0 = __low2float(h), r1 = __high2float(h);
        float p = r0 * r0 + r1 * r1;                     // this lane's part of ||y'_j||^2
        p += __shfl_xor_sync(FULL, p, 1);
        p += __shfl_xor_sync(FULL, p, 2);
        yn[j] = p;                                       // query q0 + g
    }
    for (int ct = 0; ct < 16; ct++) {
        const int clo = ct * 16 + g, chi = clo + 8;
        uint32_t out[4][M1 / 2];                         // (clo, 2tg), (clo, 2tg+1), (chi, 2tg), (chi, 2tg+1)
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
        for (int j = 0; j < M1; j++) {
            // A fragment: centroids clo and chi, coordinates 2tg, 2tg + 1 of sub-space j
            uint32_t a0 = 0, a1 = 0;
            if (tg == 0) {
                a0 = *reinterpret_cast<const uint32_t *>(cb2 + clo * M1 + j);
                a1 = *reinterpret_cast<const uint32_t *>(cb2 + chi * M1 + j);
            } else if (tg == 1) {
                a0 = pack_half2(__half2float(cb1[clo * M1 + j]), 0.f);
                a1 = pack_half2(__half2float(cb1[chi * M1 + j]), 0.f);
            }
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
            asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, "
                         "{%0, %1, %2, %3};"
                         : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
                         : "r"(a0), "r"(a1), "r"(bf[j]));
            // centroid norms (FP32 of the rounded values), summed over the quad's lanes
            const __half2 hl = *reinterpret_cast<const __half2 *>(&a0), hh = *reinterpret_cast<const __half2 *>(&a1);
            float nl = __low2float(hl) * __low2float(hl) + __high2float(hl) * __high2float(hl);
            float nh = __low2float(hh) * __low2float(hh) + __high2float(hh) * __high2float(hh);
            nl += __shfl_xor_sync(FULL, nl, 1);
            nl += __shfl_xor_sync(FULL, nl, 2);
            nh += __shfl_xor_sync(FULL, nh, 1);
            nh += __shfl_xor_sync(FULL, nh, 2);
            const float ya = __shfl_sync(FULL, yn[j], (2 * tg) * 4), yb = __shfl_sync(FULL, yn[j], (2 * tg + 1) * 4);
            const float t0 = ya + nl - 2.f * d0, t1 = yb + nl - 2.f * d1, t2 = ya + nh - 2.f * d2, t3 = yb + nh - 2.f * d3;
            // entries of consecutive sub-spaces share a 32-bit word (sub-space j - 1 low)
            if ((j & 1) == 0) {
                p0 = t0; p1 = t1; p2 = t2; p3 = t3;
            } else {
                out[0][j / 2] = pack_half2(p0, t0);
                out[1][j / 2] = pack_half2(p1, t1);
                out[2][j / 2] = pack_half2(p2, t2);
                out[3][j / 2] = pack_half2(p3, t3);
            }
        }
        // rows (query, centroid) of 32 entries = 64 bytes
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int c = e < 2 ? clo : chi;
            const int64_t q = q0 + 2 * tg + (e & 1);
            if (q >= nq) continue;
            uint4 *dst = reinterpret_cast<uint4 *>(T + (q * 256 + c) * M1);
            const uint4 *src = reinterpret_cast<const uint4 *>(&out[e][0]);
#pragma unroll
            for (int u = 0; u < 4; u++) dst[u] = src[u];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Candidates staged at a time.  Three keep a warp's staging at 2.3 KB (d = 96), so both FP32
// codebooks (192 KB) and 15 warps fit in shared memory: every codebook read is a conflict-free
// shared load.  Measured on 10k queries of the 1M workload: 0.117 ms, against 0.172 ms with
// eight staged (C2 read through L1 and L2 at 16 warps), 0.123 / 0.121 / 0.125 ms with 2 / 4 / 5
// staged (16 / 12 / 10 warps beside both codebooks).
constexpr int REF_CH = 3;

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
                // accumulated over j in order; then sum_t (y'_t - y^_t)^2 over t ascending.
                // A missing neighbour (id -1) takes weight 0: its staged rows hold stale but
                // valid codes, and fma(0, x, s) = s for the finite x of a codebook, so every
                // C2 read of the candidate is issued before the first is used (up to 4
                // coordinates per lane; beyond, the 9 x DU values would not stay in registers).
                constexpr bool HOIST = DU <= 4;
                float yh[DU], x2[HOIST ? 9 : 1][DU];
                if constexpr (HOIST) {
#pragma unroll
                    for (int j = 0; j < 9; j++) {
                        const uint8_t *c2r = st2 + (r * 9 + j) * M2P;
#pragma unroll
                        for (int u = 0; u < DU; u++) x2[j][u] = C2[(int)c2r[s2v[u]] * d + lane + 32 * u];
                    }
                }
#pragma unroll
                for (int u = 0; u < DU; u++) yh[u] = 0.f;
#pragma unroll
                for (int j = 0; j < 9; j++) {
                    const int tt = r * 9 + j;
                    const bool have = vid[tt] >= 0;
                    if (!HOIST && !have) continue;
                    const float w0 = have ? wt[r * BM * 9 + j] : 0.f;
                    const uint8_t *c1r = st1 + tt * M1, *c2r = st2 + tt * M2P;
#pragma unroll
                    for (int u = 0; u < DU; u++) {
                        const int t = lane + 32 * u;
                        if (DU == 8 && t >= d) continue;
                        // the weight of this coordinate's regression block
                        const float w = PROD ? (have ? wt[(r * BM + sbv[u]) * 9 + j] : 0.f) : w0;
                        const float x = C1s[(int)c1r[s1v[u]] * d + t] +
                                        (HOIST ? x2[HOIST ? j : 0][u] : C2[(int)c2r[s2v[u]] * d + t]);
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

static int ilog2_ceil(int64_t x);

// Automatic size (log2 entries) of the walk's shared visited table: 2^10 up to efSearch 32,
// else 2^11.  A larger table fits fewer walks per SM, and that costs more than the global
// spills it saves: on the 10M mixture at efSearch 96 / 128 / 256, 2^11 against 2^12 took
// 4.5 / 6.3 / 15.2 ms against 6.5 / 8.9 / 23.1 ms (plain level-0 launch, 20k queries) and
// 2.9 / 4.1 / 8.6 against 3.4 / 4.6 / 11.0 ms (batched beam 4, FP16 codebook).
static int auto_visited_log(int efp) { return std::min(11, std::max(10, ilog2_ceil((int64_t)efp * 32))); }

static int ilog2_ceil(int64_t x)
{
    int l = 0;
    while (((int64_t)1 << l) < x) l++;
    return l;
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

lc_status plan_search(const DeviceIndex *dv, int64_t nq, const lc_search_params *sp, SearchPlan *pl,
                      bool allow_order)
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
    P.hash_log = sp->visited_log ? sp->visited_log : auto_visited_log(P.efp);
    P.spill_log = sp->spill_log ? sp->spill_log : std::min(16, std::max(13, ilog2_ceil((int64_t)P.efp * 64)));
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
    P.tab = sp->lut_prec == LC_LUT_TABLE;
    if (P.tab && (P.variant != 2 || P.full)) {
        set_error("the table form is built for 32 level-1 sub-spaces of 3 coordinates (d = 96) and the level-1 walk");
        return LC_ERR_ARG;
    }
    P.half = sp->lut_prec == LC_LUT_FP16 || P.tab;
    cudaError_t ce;
    if (P.tab) {
        P.per_warp += (size_t)256 * TAB_M1 * 2;                 // the query's table
        P.tab_elems = (size_t)nq * 256 * TAB_M1;
        ce = walk_config_tab(wa, P.per_warp, dv->num_sms, sp->warps, &P.wpc, &P.grid, &P.smem);
    } else {
        ce = walk_config(P.half, P.variant, dv->M1, P.full, wa, P.per_warp, dv->num_sms, sp->warps, &P.wpc, &P.grid,
                         &P.smem);
    }
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
    // ordered search: worth its two extra launches once every warp takes a few queries
    P.ordered = allow_order && nq <= INT32_MAX && dv->n > 0 &&
                (sp->order == LC_ORDER_ALWAYS ||
                 (sp->order == LC_ORDER_AUTO && nq >= (int64_t)ORDER_MIN_ROUNDS * P.grid * P.wpc));
    P.ord_elems = P.ordered ? (size_t)nq * 4 : 0;
    if (P.ordered) {
        // the descent launch: its own kernel, many more warps (no level-0 state)
        WalkArgs wd{};
        wd.nq = nq;
        wd.d = dv->d;
        wd.M2P = dv->M2P;
        ce = P.tab ? descent_config_tab(wd, dv->num_sms, &P.dwpc, &P.dgrid, &P.dsmem)
                   : descent_config(P.half, P.variant, dv->M1, P.full, wd, dv->num_sms, &P.dwpc, &P.dgrid, &P.dsmem);
        if (ce != cudaSuccess) {
            set_error("descent kernel configuration failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
    }
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
    if (ce == cudaSuccess && P.tab) {
        // the batch's ADC tables on the tensor cores, from y'
        table_kernel<<<(unsigned)((nq + TAB_WARPS * 8 - 1) / (TAB_WARPS * 8)), TAB_WARPS * 32, 0, st>>>(
            sc.yq, nq, static_cast<const __half *>(dv->C1h), reinterpret_cast<__half *>(sc.tab));
        ce = cudaGetLastError();
        wa.tab = reinterpret_cast<const __half *>(sc.tab);
    }
    if (profile) cudaEventRecord(dv->ev[3], st);
    if (ce != cudaSuccess) {
        set_error("rotation kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    if (P.ordered) {
        // ordered search: the upper-level descents, the queue order, then the level-0 walks
        int32_t *seed = sc.ord, *seed_up = sc.ord + nq, *order = sc.ord + 2 * nq;
        float *seed_d = reinterpret_cast<float *>(sc.ord + 3 * nq);
        WalkArgs w1 = wa;
        w1.mode = 1;
        w1.seed = seed;
        w1.seed_up = seed_up;
        w1.seed_d = seed_d;
        ce = P.tab ? descent_run_tab(w1, P.dsmem, P.dwpc, P.dgrid, st)
                   : descent_run(P.half, P.variant, dv->M1, P.full, w1, P.dsmem, P.dwpc, P.dgrid, st);
        if (ce == cudaSuccess && cudaMemsetAsync(sc.counter, 0, sizeof(unsigned long long), st) == cudaSuccess) {
            order_kernel<<<1, ORDER_THREADS, 0, st>>>(seed_d, nq, order);
            ce = cudaGetLastError();
        } else if (ce == cudaSuccess) {
            ce = cudaGetLastError();
        }
        if (ce != cudaSuccess) {
            set_error("walk descent or queue order launch failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
        wa.mode = 2;
        wa.order = order;
        wa.seed = seed;
        wa.seed_up = seed_up;
        wa.seed_d = seed_d;
    }
    if (profile) cudaEventRecord(dv->ev[4], st);
    ce = P.tab ? walk_run_tab(wa, P.smem, P.wpc, P.grid, st)
               : walk_run(P.half, P.variant, dv->M1, P.full, wa, P.smem, P.wpc, P.grid, st);
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
    // pointer kinds: all device or all host (2: device memory of another GPU than the current
    // one, which the kernels would read through peer access or fault on)
    int cur_dev = -1;
    if (cudaGetDevice(&cur_dev) != cudaSuccess) {
        cudaGetLastError();                // no device: every pointer reads as host memory, and
        cur_dev = -1;                      // the upload below reports the missing device
    }
    auto kind = [cur_dev](const void *p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        if (at.type == cudaMemoryTypeDevice) return at.device == cur_dev ? 1 : 2;
        return at.type == cudaMemoryTypeManaged ? 1 : 0;
    };
    int kq = kind(q), ki = kind(ids), kd = kind(dists), ks = stats ? kind(stats) : kq;
    int ke = efq ? kind(efq) : kq;
    if (kq == 2 || ki == 2 || kd == 2 || ks == 2 || ke == 2) {
        set_error("device pointers must be memory of the current device (%d)", cur_dev);
        return LC_ERR_ARG;
    }
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
    rs = plan_search(dv, std::max<int64_t>(nq, 1), sp, &P, true);
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
        (P.refine && !grow(dv->shortlist, dv->sl_cap, P.sl_elems)) ||
        (P.ordered && !grow(dv->ord, dv->ord_cap, P.ord_elems)) ||
        (P.tab && !grow(dv->tab, dv->tab_cap, P.tab_elems))) {
        set_error("cudaMalloc failed for search scratch");
        return LC_ERR_OOM;
    }
    SearchScratch sc;
    sc.yq = dv->yq;
    sc.shortlist = dv->shortlist;
    sc.spill = dv->spill;
    sc.ord = dv->ord;
    sc.tab = dv->tab;
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
// file-scope array below, which every GPU that loads this library holds until exit.  Each
// query in flight gets a spill table of the size lc_search gives it at the same efSearch
// (2^13 entries up to max(ef, k) = 128, 2^14 up to 256), so a query overflows here exactly
// when it overflows in lc_search; the number of queries in flight is what the array bounds.
constexpr size_t NOALLOC_HEADER = 256;                 // counter (8 B) and status (4 B)
constexpr size_t NOALLOC_SPILL_BYTES = (size_t)64 << 20;   // 2048 tables of 2^13 entries
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + NOALLOC_SPILL_BYTES;
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
    // device memory of the current device (another GPU's memory would be read through peer
    // access, or fault), or managed memory
    auto on_device = [dev](const void *p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
    };
    if (nq > 0 && (!on_device(q) || !on_device(ids) || !on_device(dists) || (stats && !on_device(stats)))) {
        set_error("the no-allocation walk takes device pointers of the current device (%d) only", dev);
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
    // the visited tables of lc_search at this efSearch (same shared table, same spill table)
    wa.hash_log = auto_visited_log(efp);
    wa.spill_log = std::min(16, std::max(13, ilog2_ceil((int64_t)efp * 64)));
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
    ce = walk_config(false, variant, dv->M1, false, wa, per_warp, dv->num_sms, 0, &wpc, &grid, &smem);
    if (ce != cudaSuccess) {
        set_error("walk kernel configuration failed: %s", cudaGetErrorString(ce));
        return ce == cudaErrorInvalidConfiguration ? LC_ERR_CAPACITY : LC_ERR_CUDA;
    }
    // every warp in flight owns one spill table of the array
    const size_t slots = NOALLOC_SPILL_BYTES / ((size_t)4 << wa.spill_log);
    grid = (int)std::min<int64_t>(grid, (int64_t)(slots / wpc));
    // the array keeps the previous call's contents: the counter and status start at zero
    // (spill tables are cleared by the kernel before a query uses one)
    if (cudaMemsetAsync(scratch, 0, 16, st) != cudaSuccess) {
        set_error("reset of the no-allocation scratch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    ce = walk_run(false, variant, dv->M1, false, wa, smem, wpc, grid, st);
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
    extern __shared__ __align__(128) unsigned char smem_raw[];
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
    if (S < 1 || S > MERGE_MAX_SHARDS || (int64_t)S * k > MERGE_MAX) {
        set_error("need 1 <= S <= %d and S * k <= %d", MERGE_MAX_SHARDS, MERGE_MAX);
        return LC_ERR_ARG;
    }
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
    cfree(pl->sc.tab);
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
              alloc(pl->sc.yq, P.yq_elems * 4) && (!P.refine || alloc(pl->sc.shortlist, P.sl_elems * 4)) &&
              (!P.tab || alloc(pl->sc.tab, P.tab_elems * 2));
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
    // (the rotation and, in the table form, the table launch keep the largest batch: their
    // extra rows are computed and not read)
    const void *wf = P.tab ? walk_fn_tab() : walk_fn(P.half, P.variant, dv->M1, P.full);
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

lc_status profile_phases(lc_index *ix, float *rotate_ms, float *descent_ms, float *level0_ms, float *refine_ms)
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
    float r = 0, de = 0, l0 = 0, rf = 0;
    cudaEventElapsedTime(&r, dv->ev[0], dv->ev[3]);
    cudaEventElapsedTime(&de, dv->ev[3], dv->ev[4]);
    cudaEventElapsedTime(&l0, dv->ev[4], dv->ev[1]);
    if (dv->has_refine) cudaEventElapsedTime(&rf, dv->ev[1], dv->ev[2]);
    if (rotate_ms) *rotate_ms = r;
    if (descent_ms) *descent_ms = de;
    if (level0_ms) *level0_ms = l0;
    if (refine_ms) *refine_ms = rf;
    return LC_OK;
}

}  // namespace lc
