// GPU-assisted build (lc_params.build_gpu): encoding, the level-0 insertion searches and
// neighbour selections of each batch, level-0 linking and codeword assignment on the device
// copy of the index under construction, each in the host build's arithmetic where the result
// must be the host's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lc_walk.cuh"

namespace lc {

// State of the GPU-assisted build beside the device index (link0_begin .. build_gpu_end).
struct LinkDev {
    float *xh = nullptr;           // [n][d] decoded vectors
    float *adj0d = nullptr;        // [n][DEG] distance of each level-0 row entry to its owner
    int64_t n = 0;
    int64_t m = 0;                 // insertion searches in flight (build_gpu_select_start)
    int32_t *buf = nullptr;        // batch inputs: sel0 [b][DEG + 1], targets [G], starts [G + 1], src [L]
    size_t buf_cap = 0;
    int32_t *ridx = nullptr;       // rows to copy back [R]
    size_t ridx_cap = 0;
    int32_t *rid = nullptr;        // gathered rows: ids [R][DEG]
    size_t rid_cap = 0;
    // pinned host staging: selections [m][DEG + 1] or gathered rows [R][DEG], and the status word
    int32_t *h_buf = nullptr;
    size_t h_cap = 0;
    int32_t *h_status = nullptr;
};

static bool pinned_grow(LinkDev *lk, size_t need)
{
    if (!lk->h_status && cudaHostAlloc(reinterpret_cast<void **>(&lk->h_status), 16, cudaHostAllocDefault) != cudaSuccess) {
        lk->h_status = nullptr;
        return false;
    }
    if (need <= lk->h_cap && lk->h_buf) return true;
    if (lk->h_buf) cudaFreeHost(lk->h_buf);
    lk->h_buf = nullptr;
    lk->h_cap = 0;
    const size_t n = std::max<size_t>(need, 1024) + need / 4;
    if (cudaHostAlloc(reinterpret_cast<void **>(&lk->h_buf), n * 4, cudaHostAllocDefault) != cudaSuccess) {
        lk->h_buf = nullptr;
        return false;
    }
    lk->h_cap = n;
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
    if (lk->h_buf) cudaFreeHost(lk->h_buf);
    if (lk->h_status) cudaFreeHost(lk->h_status);
    delete lk;
    dv->lk = nullptr;
}


// ------------------------------------------------------------------------------------------
// GPU-assisted build.  lc_add inserts by batches, each searching the graph as it stood at the
// batch start (Section 5.1); the level-0 insertion searches of a batch are independent, so
// they run as one launch of the walk on the device copy of the index, with the exact-to-
// decoded distance of the full-decode walk (FP32); the neighbour selections and the level-0
// rows and back-links follow on the device (below).  The host keeps the upper levels of the
// batch's higher-level nodes and re-sends the upper rows a batch changed.

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

lc_status build_gpu_select_start(lc_index *ix, const float *xr, int64_t m, int efc, int32_t ep, int max_level)
{
    DeviceIndex *dv = ix->dev;
    LinkDev *lk = dv ? dv->lk : nullptr;
    if (!lk) {
        set_error("insertion searches before the build state was uploaded");
        return LC_ERR_STATE;
    }
    lk->m = 0;
    if (m <= 0) return LC_OK;
    lc_search_params sp;
    lc_default_search_params(&sp, efc, efc);
    sp.shortlist = -1;                          // the walk's own result list, sorted
    sp.walk_full = 1;
    SearchPlan P;
    // an ordered search (longest walks first) once the batch fills the GPU twice; results do not
    // depend on the order
    lc_status rs = plan_search(dv, m, &sp, &P, true);
    if (rs != LC_OK) return rs;
    if (!grow(dv->b_yq, dv->b_yq_cap, (size_t)m * dv->d) || !grow(dv->b_ids, dv->b_ids_cap, (size_t)m * efc) ||
        !grow(dv->b_d, dv->b_d_cap, (size_t)m * efc) || !grow(dv->spill, dv->spill_cap, P.spill_elems) ||
        (P.ordered && !grow(dv->ord, dv->ord_cap, P.ord_elems))) {
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
    sc.ord = dv->ord;
    sc.status = dv->status;
    sc.counter = dv->counter;
    rs = run_search(dv, P, nullptr, m, dv->b_ids, dv->b_d, nullptr, sc, 0, false, nullptr, nullptr, true);
    if (rs != LC_OK) return rs;
    // neighbour selection on the device; the selections and the status word come back into
    // pinned staging, asynchronously (build_gpu_select_finish waits for them)
    if (!grow(dv->b_sel, dv->b_sel_cap, (size_t)m * (DEG + 1)) || !pinned_grow(lk, (size_t)m * (DEG + 1))) {
        cudaGetLastError();
        set_error("allocation failed for the build's selections");
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
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(lk->h_buf, dv->b_sel, sizeof(int32_t) * m * (DEG + 1), cudaMemcpyDeviceToHost, 0) != cudaSuccess ||
        cudaMemcpyAsync(lk->h_status, dv->status, sizeof(int32_t), cudaMemcpyDeviceToHost, 0) != cudaSuccess) {
        set_error("build search failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    lk->m = m;
    return LC_OK;
}

lc_status build_gpu_select_finish(lc_index *ix, int64_t m, int32_t *sel)
{
    DeviceIndex *dv = ix->dev;
    LinkDev *lk = dv ? dv->lk : nullptr;
    if (!lk || lk->m != m) {
        set_error("no insertion searches of %lld vectors in flight", (long long)m);
        return LC_ERR_STATE;
    }
    lk->m = 0;
    if (m <= 0) return LC_OK;
    if (cudaStreamSynchronize(0) != cudaSuccess) {
        set_error("build search failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    std::memcpy(sel, lk->h_buf, sizeof(int32_t) * m * (DEG + 1));
    if (*lk->h_status) {
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

// Encoding of the vectors being added (rotation, level-1 PQ, residual, level-2 PQ), in the host
// build's float arithmetic (the rotation sums R[t][u] x_u over u in order; each centroid's
// score is ||c||^2 plus (-2 x_t) c_t over t in order; the first minimum wins; no multiply-add
// contraction), so the codes are the host's.
__global__ void rotate_exact_kernel(const float *X, int64_t n, int d, const float *RT, float *Y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int t = (int)(e - i * d);
        const float *x = X + i * d;
        float y = 0.f;
        for (int u = 0; u < d; u++) y = __fadd_rn(y, __fmul_rn(__ldg(RT + (int64_t)u * d + t), __ldg(x + u)));
        Y[e] = y;
    }
}

// codes[i][j] = argmin_c cn[j][c] + sum_t (-2 x_t) C[c][t] over sub-space j; with sub != nullptr
// the encoded vector is X minus its level-1 decode (the residual)
__global__ void pq_encode_kernel(const float *X, int64_t n, int d, int M, const uint16_t *off, const uint8_t *len,
                                 const float *C, const float *cn, uint8_t *codes, const float *C1, int M1,
                                 const uint8_t *codes1, const uint8_t *sub1)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * M; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / M;
        const int j = (int)(e - i * M), o = off[j], L = len[j];
        float m2x[16];
        for (int t = 0; t < L; t++) {
            float x = __ldg(X + i * d + o + t);
            if (codes1) x = __fsub_rn(x, __ldg(C1 + (int)codes1[i * M1 + sub1[o + t]] * d + o + t));
            m2x[t] = -2.f * x;
        }
        int best = 0;
        float bv = 0.f;
        for (int c = 0; c < 256; c++) {
            float acc = __ldg(cn + j * 256 + c);
            for (int t = 0; t < L; t++) acc = __fadd_rn(acc, __fmul_rn(m2x[t], __ldg(C + c * d + o + t)));
            if (c == 0 || acc < bv) { bv = acc; best = c; }
        }
        codes[e] = (uint8_t)best;
    }
}

lc_status build_gpu_encode(lc_index *ix, const float *x, int64_t n, float *xr, uint8_t *c1, uint8_t *c2)
{
    const int d = ix->p.d, M1 = ix->p.M1, M2 = ix->p.M2;
    std::vector<int> o1, l1, o2, l2;
    splits(d, M1, o1, l1);
    splits(d, M2, o2, l2);
    for (int j = 0; j < M2; j++)
        if (l2[j] > 16 || (j < M1 && l1[j] > 16)) {
            set_error("device encoding needs sub-spaces of at most 16 dimensions");
            return LC_ERR_ARG;
        }
    // transposed rotation and squared centroid norms exactly as the host computes them
    std::vector<float> RT((size_t)d * d), cn1((size_t)M1 * 256, 0.f), cn2((size_t)M2 * 256, 0.f);
    for (int t = 0; t < d; t++)
        for (int u = 0; u < d; u++) RT[(size_t)u * d + t] = ix->R[(size_t)t * d + u];
    auto norms = [&](const std::vector<float> &C, int M, const std::vector<int> &o, const std::vector<int> &l,
                     std::vector<float> &cn) {
        for (int j = 0; j < M; j++)
            for (int c = 0; c < 256; c++)
                for (int t = 0; t < l[j]; t++) {
                    const float v = C[(size_t)c * d + o[j] + t];
                    cn[(size_t)j * 256 + c] += v * v;
                }
    };
    norms(ix->C1, M1, o1, l1, cn1);
    norms(ix->C2, M2, o2, l2, cn2);
    std::vector<uint16_t> off1(o1.begin(), o1.end()), off2(o2.begin(), o2.end());
    std::vector<uint8_t> len1(l1.begin(), l1.end()), len2(l2.begin(), l2.end()), sub1(d);
    for (int j = 0; j < M1; j++) for (int t = o1[j]; t < o1[j] + l1[j]; t++) sub1[t] = (uint8_t)j;
    float *dRT = nullptr, *dC1 = nullptr, *dC2 = nullptr, *dcn1 = nullptr, *dcn2 = nullptr, *dX = nullptr, *dY = nullptr;
    uint16_t *doff1 = nullptr, *doff2 = nullptr;
    uint8_t *dlen1 = nullptr, *dlen2 = nullptr, *dsub1 = nullptr, *dc1 = nullptr, *dc2 = nullptr;
    const int64_t CH = std::min<int64_t>(n, 1 << 20);
    bool ok = dupload(dRT, RT) && dupload(dC1, ix->C1) && dupload(dC2, ix->C2) && dupload(dcn1, cn1) &&
              dupload(dcn2, cn2) && dupload(doff1, off1) && dupload(doff2, off2) && dupload(dlen1, len1) &&
              dupload(dlen2, len2) && dupload(dsub1, sub1) &&
              cudaMalloc(&dX, sizeof(float) * CH * d + 16) == cudaSuccess &&
              cudaMalloc(&dY, sizeof(float) * CH * d + 16) == cudaSuccess &&
              cudaMalloc(&dc1, (size_t)CH * M1 + 16) == cudaSuccess && cudaMalloc(&dc2, (size_t)CH * M2 + 16) == cudaSuccess;
    lc_status rs = LC_OK;
    if (!ok) {
        set_error("device allocation for encoding failed");
        rs = LC_ERR_OOM;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, sms) * 8;
    for (int64_t a = 0; a < n && rs == LC_OK; a += CH) {
        const int64_t m = std::min(CH, n - a);
        if (cudaMemcpy(dX, x + a * d, sizeof(float) * m * d, cudaMemcpyHostToDevice) != cudaSuccess) {
            rs = LC_ERR_CUDA;
            break;
        }
        rotate_exact_kernel<<<grid, 256>>>(dX, m, d, dRT, dY);
        pq_encode_kernel<<<grid, 256>>>(dY, m, d, M1, doff1, dlen1, dC1, dcn1, dc1, nullptr, 0, nullptr, nullptr);
        pq_encode_kernel<<<grid, 256>>>(dY, m, d, M2, doff2, dlen2, dC2, dcn2, dc2, dC1, M1, dc1, dsub1);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(xr + a * d, dY, sizeof(float) * m * d, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(c1 + a * M1, dc1, (size_t)m * M1, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(c2 + a * M2, dc2, (size_t)m * M2, cudaMemcpyDeviceToHost) != cudaSuccess)
            rs = LC_ERR_CUDA;
    }
    if (rs == LC_ERR_CUDA) set_error("encoding on the device failed: %s", cudaGetErrorString(cudaGetLastError()));
    for (void *p : {(void *)dRT, (void *)dC1, (void *)dC2, (void *)dcn1, (void *)dcn2, (void *)dX, (void *)dY,
                    (void *)doff1, (void *)doff2, (void *)dlen1, (void *)dlen2, (void *)dsub1, (void *)dc1, (void *)dc2})
        cfree(p);
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
        link0_free(dv);
    }
    ix->dev_dirty = true;                       // codewords are assigned after the graph
}

// ------------------------------------------------------------------------------------------
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
        const float dj = __shfl_sync(FULL, dist, j);
        const int32_t ij = __shfl_sync(FULL, id, j);
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
        if (__ballot_sync(FULL, id == x)) continue;      // already linked
        const float kd = l2_decoded(xt, a.xh + (int64_t)x * a.d, a.d);
        const bool valid = id >= 0;
        const int n = __popc(__ballot_sync(FULL, valid));
        const int pos = __popc(__ballot_sync(FULL, valid && key_less(dd, id, kd, x)));
        // the n + 1 candidates in order: entries before pos, the new one, the rest moved up
        const int32_t up_id = __shfl_up_sync(FULL, id, 1);
        const float up_d = __shfl_up_sync(FULL, dd, 1);
        const int32_t cid = lane < pos ? id : lane == pos ? x : up_id;
        const float cd = lane < pos ? dd : lane == pos ? kd : up_d;
        if (n < DEG) {
            id = cid;
            dd = cd;
            continue;
        }
        // DEG + 1 candidates: the last is the displaced entry DEG - 1, or the new one
        const int32_t last_id = pos == DEG ? x : __shfl_sync(FULL, id, DEG - 1);
        const float last_d = pos == DEG ? kd : __shfl_sync(FULL, dd, DEG - 1);
        int kept = 0;
        int32_t kid = -1;                                    // lane u: the u-th kept entry
        float kdd = 0.f;
        for (int c = 0; c <= DEG && kept < DEG; c++) {
            const int32_t sid = c < DEG ? __shfl_sync(FULL, cid, c) : last_id;
            const float sd = c < DEG ? __shfl_sync(FULL, cd, c) : last_d;
            const bool closer = lane < kept && l2_decoded(a.xh + (int64_t)sid * a.d, a.xh + (int64_t)kid * a.d, a.d) < sd;
            if (__ballot_sync(FULL, closer) == 0) {
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

__global__ void gather_rows_kernel(const int32_t *adj0, const int32_t *ridx, int64_t R, int32_t *rid)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R * DEG; i += (int64_t)gridDim.x * blockDim.x)
        rid[i] = adj0[(int64_t)__ldg(ridx + i / DEG) * DEG + i % DEG];
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
    if (!grow(lk->buf, lk->buf_cap, nbuf) || !grow(lk->ridx, lk->ridx_cap, (size_t)R) ||
        !grow(lk->rid, lk->rid_cap, (size_t)R * DEG) || !pinned_grow(lk, (size_t)R * DEG)) {
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
    gather_rows_kernel<<<std::max(grid, 1), 256>>>(dv->adj0, lk->ridx, R, lk->rid);
    // the ids come back (the host searches of later batches read them); the row distances
    // stay on the device until build_gpu_link0_end
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(lk->h_buf, lk->rid, (size_t)R * DEG * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("level-0 linking failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    for (int64_t r = 0; r < R; r++)
        std::memcpy(ix->adj0.data() + (int64_t)rows[r] * DEG, lk->h_buf + r * DEG, DEG * 4);
    return LC_OK;
}

lc_status build_gpu_link0_end(lc_index *ix)
{
    DeviceIndex *dv = ix->dev;
    LinkDev *lk = dv ? dv->lk : nullptr;
    if (!lk) return LC_OK;
    if (cudaMemcpy(ix->adj0_d.data(), lk->adj0d, sizeof(float) * (size_t)lk->n * DEG, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("download of the level-0 row distances failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------------------
// Regression-codebook training (Section 4.3) on the device: the assignment steps of the
// k-means that initialises the codewords and of the EM that refines them, each in the host
// build's double arithmetic (every product and sum rounded on its own, in the host's order,
// first minimum), so the assignments, and with the host's sums the codebook, are the host's.

struct EmDev {
    int device = -1;
    int64_t n = 0;
    int dim = 0;
    double *X = nullptr;           // [n][dim] points of the k-means
    double *ne = nullptr;          // [n][55] normal equations: A (45, packed upper triangle), b (9), xx
    double *C = nullptr;           // [K][dim] centres, or [K][9] codewords
    double *cn = nullptr;          // [K] squared centre norms
    size_t c_cap = 0, cn_cap = 0;
    int32_t *as = nullptr;         // [n]
    double *dm = nullptr;          // [n]
};

// as[i] = argmin_c cn[c] + sum_t (-2 x_t) C[c][t] (t in order, first minimum); dm[i] = the
// squared distance to that centre, sum over t in order.
__global__ void em_nearest_kernel(const double *X, int64_t n, int dim, const double *C, const double *cn, int K,
                                  int32_t *as, double *dm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *x = X + i * dim;
    double m2x[16];
    for (int t = 0; t < dim; t++) m2x[t] = __dmul_rn(-2.0, __ldg(x + t));
    int best = 0;
    double bv = 0.0;
    for (int c = 0; c < K; c++) {
        double acc = __ldg(cn + c);
        for (int t = 0; t < dim; t++) acc = __dadd_rn(acc, __dmul_rn(m2x[t], __ldg(C + (int64_t)c * dim + t)));
        if (c == 0 || acc < bv) { bv = acc; best = c; }
    }
    double s = 0.0;
    for (int t = 0; t < dim; t++) {
        const double df = __dsub_rn(__ldg(x + t), __ldg(C + (int64_t)best * dim + t));
        s = __dadd_rn(s, __dmul_rn(df, df));
    }
    as[i] = best;
    dm[i] = s;
}

// as[s] = argmin_c ||x - beta_c^T G||^2 = xx - 2 beta.b + beta^T A beta over codewords
// B [K][9], accumulated in the host's order (first minimum).
__global__ void em_assign_kernel(const double *ne, int64_t n, const double *B, int K, int32_t *as)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double *e = ne + s * 55;
    int best = 0;
    double bl = __longlong_as_double(0x7ff0000000000000ll);               // +inf
    for (int c = 0; c < K; c++) {
        const double *be = B + (int64_t)c * 9;
        double l = __ldg(e + 54);
        int u = 0;
        for (int p = 0; p < 9; p++) {
            const double bp = __ldg(be + p);
            l = __dsub_rn(l, __dmul_rn(__dmul_rn(2.0, bp), __ldg(e + 45 + p)));
            l = __dadd_rn(l, __dmul_rn(__dmul_rn(bp, bp), __ldg(e + u)));
            u++;
            for (int q = p + 1; q < 9; q++, u++)
                l = __dadd_rn(l, __dmul_rn(__dmul_rn(__dmul_rn(2.0, bp), __ldg(be + q)), __ldg(e + u)));
        }
        if (l < bl) { bl = l; best = c; }
    }
    as[s] = best;
}

void em_free(EmDev *em)
{
    if (!em) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (em->device >= 0) cudaSetDevice(em->device);
    cfree(em->X); cfree(em->ne); cfree(em->C); cfree(em->cn); cfree(em->as); cfree(em->dm);
    if (cur >= 0) cudaSetDevice(cur);
    delete em;
}

EmDev *em_begin(const double *X, int64_t n, int dim, const double *ne55)
{
    if (n <= 0 || dim > 16) return nullptr;
    EmDev *em = new EmDev();
    if (cudaGetDevice(&em->device) != cudaSuccess) { cudaGetLastError(); delete em; return nullptr; }
    em->n = n;
    em->dim = dim;
    bool ok = cudaMalloc(&em->X, sizeof(double) * (size_t)n * dim) == cudaSuccess &&
              cudaMalloc(&em->ne, sizeof(double) * (size_t)n * 55) == cudaSuccess &&
              cudaMalloc(&em->as, sizeof(int32_t) * (size_t)n) == cudaSuccess &&
              cudaMalloc(&em->dm, sizeof(double) * (size_t)n) == cudaSuccess &&
              cudaMemcpy(em->X, X, sizeof(double) * (size_t)n * dim, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(em->ne, ne55, sizeof(double) * (size_t)n * 55, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        em_free(em);
        return nullptr;
    }
    return em;
}

bool em_nearest(EmDev *em, const double *C, const double *cn, int K, int32_t *as, double *dm)
{
    if (!em || K < 1) return false;
    if (!grow(em->C, em->c_cap, (size_t)K * em->dim) || !grow(em->cn, em->cn_cap, (size_t)K) ||
        cudaMemcpy(em->C, C, sizeof(double) * (size_t)K * em->dim, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(em->cn, cn, sizeof(double) * (size_t)K, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    em_nearest_kernel<<<(unsigned)((em->n + 127) / 128), 128>>>(em->X, em->n, em->dim, em->C, em->cn, K, em->as, em->dm);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(as, em->as, sizeof(int32_t) * (size_t)em->n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(dm, em->dm, sizeof(double) * (size_t)em->n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

bool em_assign(EmDev *em, const double *B, int K, int32_t *as)
{
    if (!em || K < 1) return false;
    if (!grow(em->C, em->c_cap, (size_t)K * 9) ||
        cudaMemcpy(em->C, B, sizeof(double) * (size_t)K * 9, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    em_assign_kernel<<<(unsigned)((em->n + 127) / 128), 128>>>(em->ne, em->n, em->C, K, em->as);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(as, em->as, sizeof(int32_t) * (size_t)em->n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace lc
