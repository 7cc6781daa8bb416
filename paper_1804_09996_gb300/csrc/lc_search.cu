// GPU search path of Link and Code (Douze, Sablayrolles, Jegou, CVPR 2018), sm_103a.
//
// walk_kernel  (one warp per query, persistent over the query list)
//   - rotation y' = R y and the per-query ADC tables LUT[j][c] = ||y'^j - C1_j[c]||^2
//     (Section 4.1 "asymmetric distance computations"), FP32 in shared memory;
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
// FP32 walk distance: lane l holds the table entry of sub-space l (M1 = 32), of l mod 16
// (M1 = 16) or the sum of sub-spaces l and l + 32 (M1 = 64); the 32 lane values are added
// pairwise, lanes differing in bit 4 first, then bits 3, 2, 1, 0.  The sum order is the same
// for every node, so a node's distance does not depend on where it is scored.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "lc_internal.h"

namespace lc {

#define FULL 0xffffffffu

struct DeviceIndex {
    int device = -1;
    int64_t n = 0;
    int d = 0, M1 = 0, M2 = 0, max_level = 0;
    int32_t ep = -1;
    float *Rt = nullptr;          // [d][d], Rt[u*d + t] = R[t][u]
    float *C1 = nullptr, *C2 = nullptr, *B = nullptr;
    uint8_t *codes1 = nullptr, *codes2 = nullptr, *beta = nullptr;
    int32_t *adj0 = nullptr, *upper_off = nullptr, *upper_adj = nullptr;
    // scratch, grown on demand
    float *yq = nullptr; size_t yq_cap = 0;
    int32_t *shortlist = nullptr; size_t sl_cap = 0;
    int32_t *spill = nullptr; size_t spill_cap = 0;
    int32_t *status = nullptr;
    // staging for host-pointer calls
    float *q_st = nullptr; size_t q_cap = 0;
    int32_t *ids_st = nullptr; float *d_st = nullptr; int32_t *s_st = nullptr; size_t out_cap = 0;
    // profiling
    bool profile = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ev_valid = false, has_refine = false;
    int num_sms = 0;
};

static void cfree(void *p) { if (p) cudaFree(p); }

void device_free(DeviceIndex *dv)
{
    if (!dv) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (dv->device >= 0) cudaSetDevice(dv->device);
    cfree(dv->Rt); cfree(dv->C1); cfree(dv->C2); cfree(dv->B);
    cfree(dv->codes1); cfree(dv->codes2); cfree(dv->beta);
    cfree(dv->adj0); cfree(dv->upper_off); cfree(dv->upper_adj);
    cfree(dv->yq); cfree(dv->shortlist); cfree(dv->spill); cfree(dv->status);
    cfree(dv->q_st); cfree(dv->ids_st); cfree(dv->d_st); cfree(dv->s_st);
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
    int64_t nq;
    int d;
    const float *Rt, *C1;
    const uint8_t *codes1;
    const int32_t *adj0, *upper_off, *upper_adj;
    int32_t ep;
    int max_level;
    int efp;          // ef' = max(ef, k)
    int efcap;        // efp rounded up to a multiple of 32
    int R;            // shortlist length (refine) or k (no refinement)
    int refine;
    int hash_log;     // shared-memory visited table: 2^hash_log entries
    int spill_log;    // global spill table per warp: 2^spill_log entries
    int32_t *spill;
    float *yq_out;
    int32_t *short_out;
    int32_t *ids_out;
    float *dists_out;
    int32_t *stats_out;
    int32_t *status;
    SplitTab s1;
};

constexpr int MAX_WARPS_PER_BLOCK = 2;   // 1 when two warps' shared memory does not fit

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-warp shared-memory layout of the walk kernel.
struct WalkSmem {
    size_t lut, yq, stage, wkey, wflag, cand, slot, hash, total;
};

__host__ __device__ inline WalkSmem walk_smem(int M1, int d, int efcap, int hash_log)
{
    WalkSmem s;
    size_t o = 0;
    int H = M1 > 32 ? 2 : 1;
    s.lut = o;   o += (size_t)H * 256 * 32 * 4;
    s.yq = o;    o += align_up((size_t)d * 4, 16);
    s.stage = o; o += (size_t)32 * (M1 < 32 ? 16 : M1) * (M1 < 32 ? 2 : 1);
    o = align_up(o, 16);
    s.wkey = o;  o += (size_t)2 * efcap * 8;
    s.wflag = o; o += align_up((size_t)2 * efcap, 16);
    s.cand = o;  o += 32 * 8;
    s.slot = o;  o += 32 * 4;
    s.hash = o;  o += ((size_t)1 << hash_log) * 4;
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

// Bitonic sort of one 64-bit key per lane, ascending across lanes.
__device__ __forceinline__ uint64_t warp_sort64(uint64_t key, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t o = shfl_xor64(key, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            uint64_t mn = o < key ? o : key, mx = o < key ? key : o;
            key = (lower == up) ? mn : mx;
        }
    }
    return key;
}

// Reduce-scatter of v[32] (lane l holds the contribution of lane l to slots 0..31): on
// return v[0] of lane i is the sum over lanes of slot i, added lanes-differing-in-bit-4
// first, then 3, 2, 1, 0.
__device__ __forceinline__ float transpose_reduce(float (&v)[32], int lane)
{
#pragma unroll
    for (int i = 0; i < 16; i++) {
        bool hi = lane & 16;
        float send = hi ? v[i] : v[i + 16];
        float keep = hi ? v[i + 16] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        bool hi = lane & 8;
        float send = hi ? v[i] : v[i + 8];
        float keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        bool hi = lane & 4;
        float send = hi ? v[i] : v[i + 4];
        float keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        bool hi = lane & 2;
        float send = hi ? v[i] : v[i + 2];
        float keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 2);
    }
    {
        bool hi = lane & 1;
        float send = hi ? v[0] : v[1];
        float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(FULL, send, 1);
    }
    return v[0];
}

// Walk distances of up to 32 nodes: slot i holds node `e` of lane i (e < 0: empty slot, its
// result is meaningless).  Code rows are staged in shared memory, each lane then reads the
// table entries of its own sub-space(s) for every slot (conflict-free: lane l always hits
// bank l), and the slot sums are formed by transpose_reduce.
template <int M1>
__device__ __forceinline__ float score_slots(const float *lut, uint8_t *stage, const uint8_t *codes1,
                                             int32_t e, unsigned valid, int lane)
{
    if (e >= 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(codes1 + (int64_t)e * M1);
        uint4 *dst = reinterpret_cast<uint4 *>(stage + lane * M1);
#pragma unroll
        for (int u = 0; u < M1 / 16; u++) dst[u] = __ldg(src + u);
    }
    __syncwarp();
    float v[32];
    if (M1 == 32) {
#pragma unroll
        for (int i = 0; i < 32; i++) {
            v[i] = 0.f;
            if (valid & (1u << i)) {
                int c = stage[i * 32 + lane];
                v[i] = lut[c * 32 + lane];
            }
        }
    } else if (M1 == 64) {
#pragma unroll
        for (int i = 0; i < 32; i++) {
            v[i] = 0.f;
            if (valid & (1u << i)) {
                int c0 = stage[i * 64 + lane];
                int c1 = stage[i * 64 + 32 + lane];
                v[i] = lut[c0 * 32 + lane] + lut[(256 + c1) * 32 + lane];
            }
        }
    } else {   // M1 == 16: half-warp g takes the odd (g = 1) or even (g = 0) slots
        int g = lane >> 4, j = lane & 15;
#pragma unroll
        for (int s = 0; s < 16; s++) {
            int i = 2 * s + g;
            float t = 0.f;
            if (valid & (1u << i)) {
                int c = stage[i * 16 + j];
                t = lut[c * 32 + lane];
            }
            v[2 * s] = g == 0 ? t : 0.f;
            v[2 * s + 1] = g == 1 ? t : 0.f;
        }
    }
    float r = transpose_reduce(v, lane);
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

template <int M1>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * 32) walk_kernel(const WalkArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WalkSmem L = walk_smem(M1, a.d, a.efcap, a.hash_log);
    unsigned char *base = smem_raw + (size_t)warp * L.total;
    float *lut = reinterpret_cast<float *>(base + L.lut);
    float *yq = reinterpret_cast<float *>(base + L.yq);
    uint8_t *stage = base + L.stage;
    uint64_t *wkey = reinterpret_cast<uint64_t *>(base + L.wkey);
    uint8_t *wflag = base + L.wflag;
    uint64_t *cand = reinterpret_cast<uint64_t *>(base + L.cand);
    int32_t *slot = reinterpret_cast<int32_t *>(base + L.slot);
    int32_t *hash = reinterpret_cast<int32_t *>(base + L.hash);
    const int d = a.d, H = 1 << a.hash_log;
    const int wpb = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * wpb + warp;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    int32_t *spill = a.spill + (gwarp << a.spill_log);

    for (int64_t q = gwarp; q < a.nq; q += nwarps) {
        // rotation y' = R y (fixed order u = 0..d-1), kept in shared memory
        const float *y = a.Q + q * d;
        for (int t = lane; t < d; t += 32) {
            float s = 0.f;
            for (int u = 0; u < d; u++) s = fmaf(__ldg(a.Rt + (int64_t)u * d + t), __ldg(y + u), s);
            yq[t] = s;
        }
        for (int i = lane; i < H; i += 32) hash[i] = -1;
        __syncwarp();
        // ADC tables in difference form
        if (M1 == 16) {
            int g = lane >> 4, j = lane & 15;
            int o = a.s1.off[j], l = a.s1.len[j];
            for (int c = g; c < 256; c += 2) {
                float s = 0.f;
                for (int t = 0; t < l; t++) {
                    float df = yq[o + t] - __ldg(a.C1 + (int64_t)c * d + o + t);
                    s = fmaf(df, df, s);
                }
                lut[c * 32 + j] = s;
                lut[c * 32 + 16 + j] = s;
            }
        } else {
#pragma unroll
            for (int h = 0; h < M1 / 32; h++) {
                int j = h * 32 + lane;
                int o = a.s1.off[j], l = a.s1.len[j];
                for (int c = 0; c < 256; c++) {
                    float s = 0.f;
                    for (int t = 0; t < l; t++) {
                        float df = yq[o + t] - __ldg(a.C1 + (int64_t)c * d + o + t);
                        s = fmaf(df, df, s);
                    }
                    lut[(h * 256 + c) * 32 + lane] = s;
                }
            }
        }
        __syncwarp();

        // greedy descent of the upper levels
        int32_t n_up = 0, n_dist = 0, n_expand = 0;
        int32_t cur = a.ep;
        float dcur = score_slots<M1>(lut, stage, a.codes1, lane == 0 ? cur : -1, 1u, lane);
        dcur = __shfl_sync(FULL, dcur, 0);
        if (a.max_level >= 1) n_up = 1;
        for (int l = a.max_level; l >= 1; l--) {
            for (;;) {
                int32_t e = a.upper_adj[((int64_t)a.upper_off[cur] + l - 1) * DEG + lane];
                unsigned vm = __ballot_sync(FULL, e >= 0);
                n_up += __popc(vm);
                float de = score_slots<M1>(lut, stage, a.codes1, e, vm, lane);
                uint64_t k = e >= 0 ? make_key(de, e) : ~0ull;
                uint64_t best = warp_min64(k);
                if (best < make_key(dcur, cur)) {
                    cur = key_id(best);
                    dcur = key_dist(best);
                } else {
                    break;
                }
            }
        }

        // level 0: best-first search with result list W (sorted keys + expanded flags)
        int buf = 0, wn = 1;
        bool spilled = false;
        bool failed = false;
        if (lane == 0) {
            wkey[0] = make_key(dcur, cur);
            wflag[0] = 0;
            hash[hash32(cur) & (H - 1)] = cur;
        }
        n_dist = 1;
        int32_t hcount = 1, scount = 0;
        __syncwarp();
        int scan_from = 0;
        for (;;) {
            uint64_t *W = wkey + buf * a.efcap;
            uint8_t *F = wflag + buf * a.efcap;
            int pos = -1;
            for (int b0 = scan_from; b0 < wn; b0 += 32) {
                int p = b0 + lane;
                bool un = p < wn && !F[p];
                unsigned m = __ballot_sync(FULL, un);
                if (m) { pos = b0 + __ffs(m) - 1; break; }
            }
            if (pos < 0) break;
            uint64_t ckey = W[pos];
            __syncwarp();
            if (lane == 0) F[pos] = 1;
            __syncwarp();
            n_expand++;
            int32_t c = key_id(ckey);
            int32_t e = a.adj0[(int64_t)c * DEG + lane];
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
            bool fresh = e >= 0 && visit(e, hash, a.hash_log, spilled, spill, a.spill_log);
            unsigned fm = __ballot_sync(FULL, fresh);
            int nf = __popc(fm);
            n_dist += nf;
            if (spilled) scount += nf; else hcount += nf;
            if (nf == 0) { scan_from = pos; continue; }
            // compact the fresh nodes into slots 0..nf-1
            if (fresh) slot[__popc(fm & ((1u << lane) - 1))] = e;
            __syncwarp();
            int32_t se = lane < nf ? slot[lane] : -1;
            unsigned vm = nf == 32 ? FULL : ((1u << nf) - 1);
            float de = score_slots<M1>(lut, stage, a.codes1, se, vm, lane);
            uint64_t k = se >= 0 ? make_key(de, se) : ~0ull;
            if (wn == a.efp && k >= W[wn - 1]) k = ~0ull;      // cannot enter W
            unsigned km = __ballot_sync(FULL, k != ~0ull);
            int nc = __popc(km);
            if (nc == 0) { scan_from = pos; continue; }
            k = warp_sort64(k, lane);
            cand[lane] = k;
            __syncwarp();
            // merge W (wn keys) with the nc candidates into the other buffer, keep efp
            uint64_t *W2 = wkey + (buf ^ 1) * a.efcap;
            uint8_t *F2 = wflag + (buf ^ 1) * a.efcap;
            int wn2 = min(a.efp, wn + nc);
            int first_new = a.efp;
            for (int p = lane; p < wn; p += 32) {
                uint64_t key = W[p];
                int lo = 0, hi = nc;                     // candidates below key
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (cand[mid] < key) lo = mid + 1; else hi = mid;
                }
                int np = p + lo;
                if (np < wn2) { W2[np] = key; F2[np] = F[p]; }
            }
            if (lane < nc) {
                int lo = 0, hi = wn;                     // W members below the candidate
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (W[mid] < k) lo = mid + 1; else hi = mid;
                }
                int np = lane + lo;
                if (np < wn2) { W2[np] = k; F2[np] = 0; }
                if (lane == 0) first_new = np;
            }
            first_new = __shfl_sync(FULL, first_new, 0);
            // everything before the expanded node's new place, other than new candidates,
            // was already expanded
            int shifted = pos;                           // pos + (candidates below ckey)
            {
                int lo = 0, hi = nc;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (cand[mid] < ckey) lo = mid + 1; else hi = mid;
                }
                shifted = pos + lo;
            }
            scan_from = min(first_new, shifted);
            scan_from -= scan_from % 32;
            wn = wn2;
            buf ^= 1;
            __syncwarp();
        }

        // outputs
        const uint64_t *W = wkey + buf * a.efcap;
        if (a.refine) {
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
    int R, k, d, M1, M2;
    const float *C1, *C2, *B;
    const uint8_t *codes1, *codes2, *beta;
    const int32_t *adj0;
    int32_t *ids_out;
    float *dists_out;
    uint8_t sub1[256], sub2[256];   // sub-space of each dimension, per level
};

constexpr int REF_CH = 8;            // candidates staged at a time
constexpr int REF_WARPS = 4;

__host__ __device__ inline size_t refine_smem(int M1, int M2, int R)
{
    int RP = 32;
    while (RP < R) RP <<= 1;
    size_t o = 0;
    o += (size_t)REF_CH * 9 * 4;            // vertex ids
    o += (size_t)REF_CH * 9 * 4;            // weights
    o += align_up((size_t)REF_CH * 9 * M1, 16);
    o += align_up((size_t)REF_CH * 9 * M2, 16);
    o += (size_t)RP * 8;                     // keys
    return align_up(o, 128);
}

__global__ void __launch_bounds__(REF_WARPS * 32) refine_kernel(const RefineArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t per = refine_smem(a.M1, a.M2, a.R);
    unsigned char *base = smem_raw + (size_t)warp * per;
    int RP = 32;
    while (RP < a.R) RP <<= 1;
    int32_t *vid = reinterpret_cast<int32_t *>(base);
    float *wt = reinterpret_cast<float *>(base + REF_CH * 9 * 4);
    uint8_t *st1 = base + REF_CH * 9 * 8;
    uint8_t *st2 = st1 + align_up((size_t)REF_CH * 9 * a.M1, 16);
    uint64_t *keys = reinterpret_cast<uint64_t *>(st2 + align_up((size_t)REF_CH * 9 * a.M2, 16));
    const int d = a.d, M1 = a.M1, M2 = a.M2;
    const int64_t gwarp = (int64_t)blockIdx.x * REF_WARPS + warp;
    const int64_t nwarps = (int64_t)gridDim.x * REF_WARPS;

    for (int64_t q = gwarp; q < a.nq; q += nwarps) {
        const int32_t *sl = a.shortlist + q * a.R;
        int rn = 0;                                  // shortlist entries present
        for (int i = lane; i < a.R; i += 32) rn += sl[i] >= 0;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) rn += __shfl_xor_sync(FULL, rn, m);
        for (int i = lane; i < RP; i += 32) keys[i] = ~0ull;
        for (int c0 = 0; c0 < rn; c0 += REF_CH) {
            int nc = min(REF_CH, rn - c0);
            // G(x) vertex ids and codeword weights: task = (candidate r, column j)
            for (int t = lane; t < nc * 9; t += 32) {
                int r = t / 9, j = t % 9;
                int32_t i = sl[c0 + r];
                int32_t v = j == 0 ? i : a.adj0[(int64_t)i * DEG + j - 1];
                vid[t] = v;
                wt[t] = __ldg(a.B + (int)a.beta[i] * 9 + j);
            }
            __syncwarp();
            // stage both code rows of every vertex (row-wise, coalesced)
            for (int t = 0; t < nc * 9; t++) {
                int32_t v = vid[t];
                if (v < 0) continue;
                for (int b = lane; b < M1; b += 32) st1[t * M1 + b] = a.codes1[(int64_t)v * M1 + b];
                for (int b = lane; b < M2; b += 32) st2[t * M2 + b] = a.codes2[(int64_t)v * M2 + b];
            }
            __syncwarp();
            for (int r = 0; r < nc; r++) {
                float part = 0.f;
                for (int t = lane; t < d; t += 32) {
                    int s1 = a.sub1[t], s2 = a.sub2[t];
                    float yh = 0.f;
#pragma unroll
                    for (int j = 0; j < 9; j++) {
                        int tt = r * 9 + j;
                        if (vid[tt] < 0) continue;
                        float x = __ldg(a.C1 + (int)st1[tt * M1 + s1] * d + t) +
                                  __ldg(a.C2 + (int)st2[tt * M2 + s2] * d + t);
                        yh = fmaf(wt[tt], x, yh);
                    }
                    float df = a.yq[q * d + t] - yh;
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
            uint64_t kk = i < RP ? keys[i] : ~0ull;
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

static lc_status upload(lc_index *ix)
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
        if (cudaMalloc(&dv->status, sizeof(int32_t)) != cudaSuccess) {
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
    bool ok = dupload(dv->Rt, Rt) && dupload(dv->C1, ix->C1) && dupload(dv->C2, ix->C2) &&
              dupload(dv->B, ix->B) && dupload(dv->codes1, ix->codes1) &&
              dupload(dv->codes2, ix->codes2) && dupload(dv->beta, ix->beta) &&
              dupload(dv->adj0, ix->adj0) && dupload(dv->upper_off, off) &&
              dupload(dv->upper_adj, ix->upper_adj);
    if (!ok) {
        set_error("device upload of the index failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_OOM;
    }
    dv->n = ix->n;
    dv->d = d;
    dv->M1 = ix->p.M1;
    dv->M2 = ix->p.M2;
    dv->ep = ix->ep;
    dv->max_level = ix->max_level < 0 ? 0 : ix->max_level;
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

template <int M1>
static cudaError_t launch_walk(const WalkArgs &wa, size_t smem_per_warp, int num_sms, int *wpb_out,
                               int *grid_out)
{
    int wpb = smem_per_warp * MAX_WARPS_PER_BLOCK <= MAX_SMEM_PER_BLOCK ? MAX_WARPS_PER_BLOCK : 1;
    size_t smem = smem_per_warp * wpb;
    if (smem > MAX_SMEM_PER_BLOCK) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<M1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<M1>, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (wa.nq + wpb - 1) / wpb;
    *grid_out = (int)std::min<int64_t>(need, (int64_t)per_sm * num_sms);
    *wpb_out = wpb;
    return cudaSuccess;
}

template <int M1>
static cudaError_t run_walk(const WalkArgs &wa, size_t smem_per_warp, int wpb, int grid, cudaStream_t st)
{
    walk_kernel<M1><<<grid, wpb * 32, smem_per_warp * wpb, st>>>(wa);
    return cudaGetLastError();
}

lc_status search(lc_index *ix, const float *q, int64_t nq, const lc_search_params *sp,
                 int32_t *ids, float *dists, int32_t *stats, void *stream_)
{
    cudaStream_t st = (cudaStream_t)stream_;
    int k = sp->k, efp = std::max(sp->ef, sp->k);
    bool refine = sp->shortlist >= 0;
    int R = refine ? std::max(sp->shortlist > 0 ? sp->shortlist : 10, k) : k;
    if (refine && R > MAX_SHORTLIST) {
        set_error("shortlist %d exceeds %d", R, MAX_SHORTLIST);
        return LC_ERR_ARG;
    }
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
    if (kq != ki || kq != kd || kq != ks) {
        set_error("query and output pointers must all be host or all be device memory");
        return LC_ERR_ARG;
    }
    bool dev_ptrs = kq == 1;
    lc_status rs = upload(ix);
    if (rs != LC_OK) return rs;
    DeviceIndex *dv = ix->dev;
    if (nq == 0) return LC_OK;
    const float *dq = q;
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
        if (cudaMemcpyAsync(dv->q_st, q, sizeof(float) * nq * dv->d, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            set_error("query upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            return LC_ERR_CUDA;
        }
        dq = dv->q_st;
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

    WalkArgs wa{};
    wa.Q = dq; wa.nq = nq; wa.d = dv->d;
    wa.Rt = dv->Rt; wa.C1 = dv->C1; wa.codes1 = dv->codes1;
    wa.adj0 = dv->adj0; wa.upper_off = dv->upper_off; wa.upper_adj = dv->upper_adj;
    wa.ep = dv->ep; wa.max_level = dv->max_level;
    wa.efp = efp; wa.efcap = (int)align_up(efp, 32);
    wa.R = R; wa.refine = refine ? 1 : 0;
    wa.hash_log = sp->visited_log ? sp->visited_log : std::min(14, std::max(10, ilog2_ceil((int64_t)efp * 32)));
    wa.spill_log = 16;
    wa.status = dv->status;
    wa.stats_out = dstats;
    std::vector<int> off, len;
    splits(dv->d, dv->M1, off, len);
    for (int j = 0; j < dv->M1; j++) { wa.s1.off[j] = (uint16_t)off[j]; wa.s1.len[j] = (uint8_t)len[j]; }
    size_t per_warp = walk_smem(dv->M1, dv->d, wa.efcap, wa.hash_log).total;
    int grid = 0, wpb = 1;
    cudaError_t ce;
    if (dv->M1 == 16) ce = launch_walk<16>(wa, per_warp, dv->num_sms, &wpb, &grid);
    else if (dv->M1 == 32) ce = launch_walk<32>(wa, per_warp, dv->num_sms, &wpb, &grid);
    else ce = launch_walk<64>(wa, per_warp, dv->num_sms, &wpb, &grid);
    if (ce != cudaSuccess) {
        set_error("walk kernel configuration failed (%zu B shared memory per warp): %s", per_warp,
                  cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    size_t slots = (size_t)grid * wpb;
    if (!grow(dv->spill, dv->spill_cap, slots << wa.spill_log)) {
        set_error("cudaMalloc failed for the visited spill tables");
        return LC_ERR_OOM;
    }
    wa.spill = dv->spill;
    if (refine) {
        if (!grow(dv->yq, dv->yq_cap, (size_t)nq * dv->d) || !grow(dv->shortlist, dv->sl_cap, (size_t)nq * R)) {
            set_error("cudaMalloc failed for search scratch");
            return LC_ERR_OOM;
        }
        wa.yq_out = dv->yq;
        wa.short_out = dv->shortlist;
    } else {
        wa.ids_out = dids;
        wa.dists_out = ddists;
    }
    if (cudaMemsetAsync(dv->status, 0, sizeof(int32_t), st) != cudaSuccess) {
        set_error("status reset failed");
        return LC_ERR_CUDA;
    }
    if (dv->profile) {
        for (auto &e : dv->ev)
            if (!e) cudaEventCreate(&e);
        cudaEventRecord(dv->ev[0], st);
    }
    if (dv->M1 == 16) ce = run_walk<16>(wa, per_warp, wpb, grid, st);
    else if (dv->M1 == 32) ce = run_walk<32>(wa, per_warp, wpb, grid, st);
    else ce = run_walk<64>(wa, per_warp, wpb, grid, st);
    if (dv->profile) cudaEventRecord(dv->ev[1], st);
    if (ce != cudaSuccess) {
        set_error("walk kernel launch failed: %s", cudaGetErrorString(ce));
        return LC_ERR_CUDA;
    }
    if (refine) {
        RefineArgs ra{};
        ra.yq = dv->yq; ra.shortlist = dv->shortlist; ra.nq = nq; ra.R = R; ra.k = k; ra.d = dv->d;
        ra.M1 = dv->M1; ra.M2 = dv->M2; ra.C1 = dv->C1; ra.C2 = dv->C2; ra.B = dv->B;
        ra.codes1 = dv->codes1; ra.codes2 = dv->codes2; ra.beta = dv->beta; ra.adj0 = dv->adj0;
        ra.ids_out = dids; ra.dists_out = ddists;
        std::vector<int> o2, l2;
        splits(dv->d, dv->M1, off, len);
        splits(dv->d, dv->M2, o2, l2);
        for (int j = 0; j < dv->M1; j++) for (int t = off[j]; t < off[j] + len[j]; t++) ra.sub1[t] = (uint8_t)j;
        for (int j = 0; j < dv->M2; j++) for (int t = o2[j]; t < o2[j] + l2[j]; t++) ra.sub2[t] = (uint8_t)j;
        size_t rs_per = refine_smem(dv->M1, dv->M2, R);
        size_t rsm = rs_per * REF_WARPS;
        cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_kernel, REF_WARPS * 32, rsm);
        int64_t need = (nq + REF_WARPS - 1) / REF_WARPS;
        int rgrid = (int)std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * dv->num_sms);
        refine_kernel<<<rgrid, REF_WARPS * 32, rsm, st>>>(ra);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            set_error("refine kernel launch failed: %s", cudaGetErrorString(ce));
            return LC_ERR_CUDA;
        }
    }
    if (dv->profile) {
        cudaEventRecord(dv->ev[2], st);
        dv->ev_valid = true;
        dv->has_refine = refine;
    }
    if (!dev_ptrs) {
        cudaMemcpyAsync(ids, dids, sizeof(int32_t) * nq * k, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(dists, ddists, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st);
        if (stats) cudaMemcpyAsync(stats, dstats, sizeof(int32_t) * nq * 3, cudaMemcpyDeviceToHost, st);
        int32_t status = 0;
        cudaMemcpyAsync(&status, dv->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        ce = cudaStreamSynchronize(st);
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
