// GPU-assisted build, level-0 linking of an insertion batch (Section 5.1: the vectors are
// inserted by batches, each batch linked into the graph as it stood at the batch start).
//
// After the batch's level-0 neighbour selections are known, two kernels finish level 0 on the
// device copy of the graph:
//  * own_rows_kernel: each member's level-0 row is its selections sorted by (distance, id);
//  * links_kernel: each existing node that a member selected (a target) receives the back-link,
//    one warp per target applying its sources in increasing id: a source already in the row is
//    skipped; otherwise it is inserted in (distance, id) order, and a row that would exceed
//    DEG entries is shrunk by HNSW's heuristic (a candidate is kept unless it is closer to an
//    already kept one than to the target), kept entries in candidate order.
// The distances are the host build's decoded-to-decoded distances in its float arithmetic
// (eight partial sums over coordinate groups, then a fixed tree; no multiply-add
// contraction), read from the decoded vectors, so every row equals the host build's.  The rows
// written are copied back to the host copy, which the host-side insertions of the batch's
// higher-level nodes search.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lc_device.h"

namespace lc {

#define LK_FULL 0xffffffffu

struct LinkDev {
    float *xh = nullptr;           // [n][d] decoded vectors
    float *adj0d = nullptr;        // [n][DEG] distance of each level-0 row entry to its owner
    int64_t n = 0;
    int32_t *buf = nullptr;        // batch inputs: sel0 [b][DEG + 1], targets [G], starts [G + 1], src [L]
    size_t buf_cap = 0;
    int32_t *ridx = nullptr;       // rows to copy back [R]
    size_t ridx_cap = 0;
    int32_t *rid = nullptr;        // gathered rows: ids [R][DEG]
    size_t rid_cap = 0;
    float *rdist = nullptr;        // gathered rows: distances [R][DEG]
    size_t rdist_cap = 0;
};

template <class T>
static bool lk_grow(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t n = std::max<size_t>(need, 1) + need / 4;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return false;
    cap = n;
    return true;
}

void link0_free(DeviceIndex *dv)
{
    if (!dv || !dv->lk) return;
    LinkDev *lk = dv->lk;
    if (lk->xh) cudaFree(lk->xh);
    if (lk->adj0d) cudaFree(lk->adj0d);
    if (lk->buf) cudaFree(lk->buf);
    if (lk->ridx) cudaFree(lk->ridx);
    if (lk->rid) cudaFree(lk->rid);
    if (lk->rdist) cudaFree(lk->rdist);
    delete lk;
    dv->lk = nullptr;
}

// ||a - b||^2 of two decoded vectors in the host build's order: s_u accumulates coordinates
// t = u (mod 8) of the full groups of 8, the remaining coordinates go to s_0, then
// ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7)); every operation rounded on its own.
__device__ float l2_decoded(const float *a, const float *b, int d)
{
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int t = 0;
    if ((d & 3) == 0) {
        // rows are 16-byte aligned: two float4 loads per operand and group
        for (; t + 8 <= d; t += 8) {
            const float4 a0 = __ldg(reinterpret_cast<const float4 *>(a + t));
            const float4 a1 = __ldg(reinterpret_cast<const float4 *>(a + t + 4));
            const float4 b0 = __ldg(reinterpret_cast<const float4 *>(b + t));
            const float4 b1 = __ldg(reinterpret_cast<const float4 *>(b + t + 4));
            const float x[8] = {__fsub_rn(a0.x, b0.x), __fsub_rn(a0.y, b0.y), __fsub_rn(a0.z, b0.z),
                                __fsub_rn(a0.w, b0.w), __fsub_rn(a1.x, b1.x), __fsub_rn(a1.y, b1.y),
                                __fsub_rn(a1.z, b1.z), __fsub_rn(a1.w, b1.w)};
#pragma unroll
            for (int u = 0; u < 8; u++) s[u] = __fadd_rn(s[u], __fmul_rn(x[u], x[u]));
        }
    } else {
        for (; t + 8 <= d; t += 8) {
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const float x = __fsub_rn(__ldg(a + t + u), __ldg(b + t + u));
                s[u] = __fadd_rn(s[u], __fmul_rn(x, x));
            }
        }
    }
    for (; t < d; t++) {
        const float x = __fsub_rn(__ldg(a + t), __ldg(b + t));
        s[0] = __fadd_rn(s[0], __fmul_rn(x, x));
    }
    return __fadd_rn(__fadd_rn(__fadd_rn(s[0], s[1]), __fadd_rn(s[2], s[3])),
                     __fadd_rn(__fadd_rn(s[4], s[5]), __fadd_rn(s[6], s[7])));
}

// (distance, id) lexicographic order of the host build's keys
__device__ __forceinline__ bool key_less(float da, int32_t ia, float db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

struct Link0Args {
    const float *xh;
    int32_t *adj0;                 // [n][DEG]
    float *adj0d;                  // [n][DEG]
    int d;
    int64_t first, b;              // members first .. first + b - 1
    const int32_t *sel0;           // [b][DEG + 1]
    int64_t G;
    const int32_t *targets, *starts, *src;
};

// One warp per member: its level-0 row, the selections sorted by (distance, id) (ids distinct,
// so the ranks are distinct); entries past the count stay empty (-1, 0).
__global__ void __launch_bounds__(256) own_rows_kernel(const Link0Args a)
{
    const int lane = threadIdx.x & 31;
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= a.b) return;                                // whole warps leave together
    const int64_t x = a.first + u;
    const int32_t *s = a.sel0 + u * (DEG + 1);
    const int cnt = __ldg(s + DEG);
    int32_t id = -1;
    float dist = 0.f;
    if (lane < cnt) {
        id = __ldg(s + lane);
        dist = l2_decoded(a.xh + x * a.d, a.xh + (int64_t)id * a.d, a.d);
    }
    int rank = 0;
    for (int j = 0; j < cnt; j++) {
        const float dj = __shfl_sync(LK_FULL, dist, j);
        const int32_t ij = __shfl_sync(LK_FULL, id, j);
        rank += key_less(dj, ij, dist, id);
    }
    const int pos = lane < cnt ? rank : lane;
    a.adj0[x * DEG + pos] = id;
    a.adj0d[x * DEG + pos] = dist;
}

// One warp per target: lane s holds entry s of the row (packed: valid entries first, in
// (distance, id) order).
__global__ void __launch_bounds__(256) links_kernel(const Link0Args a)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= a.G) return;                                // whole warps leave together
    const int64_t t = __ldg(a.targets + g);
    const float *xt = a.xh + t * a.d;
    int32_t id = a.adj0[t * DEG + lane];
    float dd = a.adj0d[t * DEG + lane];
    const int i1 = __ldg(a.starts + g + 1);
    for (int i = __ldg(a.starts + g); i < i1; i++) {
        const int32_t x = __ldg(a.src + i);
        if (__ballot_sync(LK_FULL, id == x)) continue;      // already linked
        const float kd = l2_decoded(xt, a.xh + (int64_t)x * a.d, a.d);
        const bool valid = id >= 0;
        const int n = __popc(__ballot_sync(LK_FULL, valid));
        const int pos = __popc(__ballot_sync(LK_FULL, valid && key_less(dd, id, kd, x)));
        // the n + 1 candidates in order: entries before pos, the new one, the rest moved up
        const int32_t up_id = __shfl_up_sync(LK_FULL, id, 1);
        const float up_d = __shfl_up_sync(LK_FULL, dd, 1);
        const int32_t cid = lane < pos ? id : lane == pos ? x : up_id;
        const float cd = lane < pos ? dd : lane == pos ? kd : up_d;
        if (n < DEG) {
            id = cid;
            dd = cd;
            continue;
        }
        // DEG + 1 candidates: the last is the displaced entry DEG - 1, or the new one
        const int32_t last_id = pos == DEG ? x : __shfl_sync(LK_FULL, id, DEG - 1);
        const float last_d = pos == DEG ? kd : __shfl_sync(LK_FULL, dd, DEG - 1);
        int kept = 0;
        int32_t kid = -1;                                    // lane u: the u-th kept entry
        float kdd = 0.f;
        for (int c = 0; c <= DEG && kept < DEG; c++) {
            const int32_t sid = c < DEG ? __shfl_sync(LK_FULL, cid, c) : last_id;
            const float sd = c < DEG ? __shfl_sync(LK_FULL, cd, c) : last_d;
            const bool closer = lane < kept && l2_decoded(a.xh + (int64_t)sid * a.d, a.xh + (int64_t)kid * a.d, a.d) < sd;
            if (__ballot_sync(LK_FULL, closer) == 0) {
                if (lane == kept) { kid = sid; kdd = sd; }
                kept++;
            }
        }
        id = lane < kept ? kid : -1;
        dd = lane < kept ? kdd : 0.f;
    }
    a.adj0[t * DEG + lane] = id;
    a.adj0d[t * DEG + lane] = dd;
}

__global__ void gather_rows_kernel(const int32_t *adj0, const float *adj0d, const int32_t *ridx, int64_t R,
                                   int32_t *rid, float *rdist)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R * DEG; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = (int64_t)__ldg(ridx + i / DEG) * DEG + i % DEG;
        rid[i] = adj0[src];
        rdist[i] = adj0d[src];
    }
}

lc_status build_gpu_link0_begin(lc_index *ix)
{
    DeviceIndex *dv = ix->dev;
    if (!dv) {
        set_error("level-0 linking without a device index");
        return LC_ERR_STATE;
    }
    link0_free(dv);
    LinkDev *lk = new LinkDev();
    dv->lk = lk;
    const int64_t n = ix->n;
    const size_t xb = sizeof(float) * (size_t)n * ix->p.d, db = sizeof(float) * (size_t)n * DEG;
    if ((int64_t)ix->xh.size() != n * ix->p.d || (int64_t)ix->adj0_d.size() != n * DEG) {
        set_error("build state out of step with the index");
        link0_free(dv);
        return LC_ERR_STATE;
    }
    if (cudaMalloc(&lk->xh, std::max<size_t>(xb, 16)) != cudaSuccess ||
        cudaMalloc(&lk->adj0d, std::max<size_t>(db, 16)) != cudaSuccess) {
        cudaGetLastError();
        link0_free(dv);
        set_error("cudaMalloc failed for the build's decoded vectors and row distances");
        return LC_ERR_OOM;
    }
    if (cudaMemcpy(lk->xh, ix->xh.data(), xb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(lk->adj0d, ix->adj0_d.data(), db, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("upload of the build state failed: %s", cudaGetErrorString(cudaGetLastError()));
        link0_free(dv);
        return LC_ERR_CUDA;
    }
    lk->n = n;
    return LC_OK;
}

lc_status build_gpu_link0(lc_index *ix, int64_t first, int64_t b, const int32_t *sel0, const int32_t *targets,
                          const int32_t *starts, int64_t G, const int32_t *src)
{
    DeviceIndex *dv = ix->dev;
    LinkDev *lk = dv ? dv->lk : nullptr;
    if (!lk || first + b > lk->n) {
        set_error("level-0 linking before its state was uploaded");
        return LC_ERR_STATE;
    }
    if (b <= 0) return LC_OK;
    const int64_t L = G > 0 ? starts[G] : 0;
    const size_t nsel = (size_t)b * (DEG + 1), nbuf = nsel + (size_t)G + (size_t)(G + 1) + (size_t)L;
    const int64_t R = b + G;                             // rows written: the members', the targets'
    if (!lk_grow(lk->buf, lk->buf_cap, nbuf) || !lk_grow(lk->ridx, lk->ridx_cap, (size_t)R) ||
        !lk_grow(lk->rid, lk->rid_cap, (size_t)R * DEG) || !lk_grow(lk->rdist, lk->rdist_cap, (size_t)R * DEG)) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the build's level-0 linking");
        return LC_ERR_OOM;
    }
    // inputs in one buffer: sel0, targets, starts, sources; the rows to copy back
    std::vector<int32_t> h(nbuf);
    std::memcpy(h.data(), sel0, nsel * 4);
    if (G > 0) {
        std::memcpy(h.data() + nsel, targets, (size_t)G * 4);
        std::memcpy(h.data() + nsel + G, starts, (size_t)(G + 1) * 4);
        std::memcpy(h.data() + nsel + 2 * G + 1, src, (size_t)L * 4);
    }
    std::vector<int32_t> rows((size_t)R);
    for (int64_t u = 0; u < b; u++) rows[u] = (int32_t)(first + u);
    for (int64_t g = 0; g < G; g++) rows[b + g] = targets[g];
    if (cudaMemcpy(lk->buf, h.data(), nbuf * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(lk->ridx, rows.data(), (size_t)R * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("level-0 linking upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    Link0Args a{};
    a.xh = lk->xh; a.adj0 = dv->adj0; a.adj0d = lk->adj0d; a.d = ix->p.d;
    a.first = first; a.b = b; a.sel0 = lk->buf;
    a.G = G; a.targets = lk->buf + nsel; a.starts = lk->buf + nsel + G; a.src = lk->buf + nsel + 2 * G + 1;
    // members' rows first, then the back-links (disjoint rows: a member is never a target of
    // its own batch, whose searches saw the graph as it stood at the batch start)
    own_rows_kernel<<<(unsigned)((b * 32 + 255) / 256), 256>>>(a);
    if (G > 0) links_kernel<<<(unsigned)((G * 32 + 255) / 256), 256>>>(a);
    const int grid = (int)std::min<int64_t>((R * DEG + 255) / 256, (int64_t)dv->num_sms * 8);
    gather_rows_kernel<<<std::max(grid, 1), 256>>>(dv->adj0, lk->adj0d, lk->ridx, R, lk->rid, lk->rdist);
    std::vector<int32_t> rid((size_t)R * DEG);
    std::vector<float> rdist((size_t)R * DEG);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(rid.data(), lk->rid, rid.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rdist.data(), lk->rdist, rdist.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("level-0 linking failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    for (int64_t r = 0; r < R; r++) {
        std::memcpy(ix->adj0.data() + (int64_t)rows[r] * DEG, rid.data() + r * DEG, DEG * 4);
        std::memcpy(ix->adj0_d.data() + (int64_t)rows[r] * DEG, rdist.data() + r * DEG, DEG * 4);
    }
    return LC_OK;
}

}  // namespace lc
