// C ABI of liblc.so (declared in include/lc.h): argument checking, index state, import,
// export and the on-disk format.  The build lives in lc_build.cpp and the GPU search in
// lc_search.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lc_internal.h"

namespace lc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static lc_status check_params(const lc_params *p)
{
    if (!p) { set_error("params is NULL"); return LC_ERR_ARG; }
    if (p->d < 1 || p->d > 256) { set_error("d = %d outside 1..256", p->d); return LC_ERR_ARG; }
    if (p->M1 != 16 && p->M1 != 32 && p->M1 != 64) { set_error("M1 = %d must be 16, 32 or 64", p->M1); return LC_ERR_ARG; }
    if (p->M1 > p->d) { set_error("M1 = %d exceeds d = %d", p->M1, p->d); return LC_ERR_ARG; }
    if (p->M2 < 1 || p->M2 > 256 || p->M2 > p->d) { set_error("M2 = %d outside 1..min(256, d)", p->M2); return LC_ERR_ARG; }
    if (p->deg != DEG || p->deg_upper != DEG) { set_error("graph degrees must be %d", DEG); return LC_ERR_ARG; }
    if (p->level_ratio < 2) { set_error("level_ratio must be >= 2"); return LC_ERR_ARG; }
    if (p->ef_construction < 1 || p->ef_construction > 4096) { set_error("ef_construction outside 1..4096"); return LC_ERR_ARG; }
    if (p->beta_train_n < 1 || p->beta_iters < 0 || p->kmeans_iters < 0 || p->opq_iters < 0) {
        set_error("negative iteration count or empty codebook training set");
        return LC_ERR_ARG;
    }
    if (p->batch_max < 1) { set_error("batch_max must be >= 1"); return LC_ERR_ARG; }
    if (p->beta_M < 1 || p->beta_M > MAX_BETA_M || p->beta_M > p->d) {
        set_error("beta_M = %d outside 1..min(%d, d)", p->beta_M, MAX_BETA_M);
        return LC_ERR_ARG;
    }
    if (p->beta_K < 1 || p->beta_K > NBETA) { set_error("beta_K = %d outside 1..%d", p->beta_K, NBETA); return LC_ERR_ARG; }
    if (p->build_gpu != 0 && p->build_gpu != 1) { set_error("build_gpu = %d is neither 0 nor 1", p->build_gpu); return LC_ERR_ARG; }
    return LC_OK;
}

lc_status check_search_params(const lc_search_params *sp)
{
    if (sp->k < 1 || sp->k > MAX_K) { set_error("k = %d outside 1..%d", sp->k, MAX_K); return LC_ERR_ARG; }
    if (sp->ef < 1) { set_error("ef must be >= 1"); return LC_ERR_ARG; }
    if ((sp->ef > sp->k ? sp->ef : sp->k) > MAX_EF) { set_error("max(ef, k) exceeds %d", MAX_EF); return LC_ERR_ARG; }
    if (sp->shortlist > MAX_SHORTLIST) { set_error("shortlist exceeds %d", MAX_SHORTLIST); return LC_ERR_ARG; }
    if (sp->lut_prec != LC_LUT_FP32 && sp->lut_prec != LC_LUT_FP16 && sp->lut_prec != LC_LUT_TABLE) {
        set_error("unsupported lut_prec %d", sp->lut_prec);
        return LC_ERR_ARG;
    }
    if (sp->mode != LC_MODE_PLAIN && sp->mode != LC_MODE_BATCHED) { set_error("unsupported mode %d", sp->mode); return LC_ERR_ARG; }
    if (sp->mode == LC_MODE_BATCHED && (sp->beam < 2 || sp->beam > 8)) {
        set_error("beam = %d outside 2..8 for the batched mode", sp->beam);
        return LC_ERR_ARG;
    }
    if (sp->max_dist < 0) { set_error("max_dist must be >= 0"); return LC_ERR_ARG; }
    if (sp->warps < 0 || sp->warps > 16) { set_error("warps = %d outside 0..16", sp->warps); return LC_ERR_ARG; }
    if (sp->walk_full != 0 && sp->walk_full != 1) { set_error("walk_full = %d is neither 0 nor 1", sp->walk_full); return LC_ERR_ARG; }
    if (sp->order != LC_ORDER_AUTO && sp->order != LC_ORDER_NEVER && sp->order != LC_ORDER_ALWAYS) {
        set_error("order = %d is not LC_ORDER_AUTO, LC_ORDER_NEVER or LC_ORDER_ALWAYS", sp->order);
        return LC_ERR_ARG;
    }
    if (sp->visited_log != 0 && (sp->visited_log < 10 || sp->visited_log > 14)) {
        set_error("visited_log = %d outside 10..14", sp->visited_log);
        return LC_ERR_ARG;
    }
    if (sp->spill_log != 0 && (sp->spill_log < 8 || sp->spill_log > 16)) {
        set_error("spill_log = %d outside 8..16", sp->spill_log);
        return LC_ERR_ARG;
    }
    return LC_OK;
}

}  // namespace lc

using namespace lc;

extern "C" {

void lc_default_params(lc_params *p, int d, int M1, int M2)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->d = d;
    p->M1 = M1;
    p->M2 = M2;
    p->use_opq = 1;
    p->deg = DEG;
    p->deg_upper = DEG;
    p->level_ratio = 30;
    p->ef_construction = 40;
    p->beta_train_n = 250000;
    p->beta_iters = 10;
    p->kmeans_iters = 25;
    p->opq_iters = 10;
    p->batch_max = 4096;
    p->n_threads = 0;
    p->seed = 1804;
    p->beta_M = 1;
    p->beta_K = NBETA;
}

void lc_default_search_params(lc_search_params *p, int k, int ef)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k = k;
    p->ef = ef;
    p->shortlist = 0;
    p->lut_prec = LC_LUT_FP32;
    p->mode = LC_MODE_PLAIN;
    p->beam = 1;
}

lc_status lc_create(const lc_params *params, lc_index **out)
{
    set_error("");
    if (!out) { set_error("out is NULL"); return LC_ERR_ARG; }
    *out = nullptr;
    lc_status s = check_params(params);
    if (s != LC_OK) return s;
    lc_index *ix = new (std::nothrow) lc_index();
    if (!ix) { set_error("out of host memory"); return LC_ERR_OOM; }
    ix->p = *params;
    *out = ix;
    return LC_OK;
}

lc_status lc_train(lc_index *ix, const float *xt, int64_t nt)
{
    set_error("");
    if (!ix || !xt) { set_error("null index or training set"); return LC_ERR_ARG; }
    if (nt < KSUB) { set_error("need at least %d training vectors, got %lld", KSUB, (long long)nt); return LC_ERR_ARG; }
    if (ix->trained) { set_error("index is already trained"); return LC_ERR_STATE; }
    try {
        return build_train(ix, xt, nt);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory during training");
        return LC_ERR_OOM;
    }
}

lc_status lc_add(lc_index *ix, const float *x, int64_t n)
{
    set_error("");
    if (!ix || (!x && n > 0) || n < 0) { set_error("null index or vectors, or negative count"); return LC_ERR_ARG; }
    if (!ix->trained) { set_error("lc_add before lc_train"); return LC_ERR_STATE; }
    if (ix->n + n > (int64_t)0x7fffffff) { set_error("index would exceed 2^31 - 1 vectors"); return LC_ERR_ARG; }
    if (n == 0) return LC_OK;
    try {
        return build_add(ix, x, n);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory during add");
        return LC_ERR_OOM;
    }
}

lc_status lc_add_u8(lc_index *ix, const uint8_t *x, int64_t n)
{
    set_error("");
    if (!ix || (!x && n > 0) || n < 0) { set_error("null index or vectors, or negative count"); return LC_ERR_ARG; }
    std::vector<float> xf;
    try {
        xf.resize((size_t)n * ix->p.d);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory converting %lld uint8 vectors", (long long)n);
        return LC_ERR_OOM;
    }
    for (size_t i = 0; i < xf.size(); i++) xf[i] = (float)x[i];
    return lc_add(ix, xf.data(), n);
}

lc_status lc_search_ex(lc_index *ix, const void *q, int qtype, int64_t nq, const lc_search_params *sp,
                       const int32_t *ef, int32_t *ids, float *dists, int32_t *stats, void *stream)
{
    set_error("");
    if (!ix || !sp) { set_error("null index or search parameters"); return LC_ERR_ARG; }
    if (nq < 0 || (nq > 0 && (!q || !ids || !dists))) { set_error("null query or output buffer"); return LC_ERR_ARG; }
    if (qtype != LC_QUERY_F32 && qtype != LC_QUERY_U8) { set_error("query type %d is neither LC_QUERY_F32 nor LC_QUERY_U8", qtype); return LC_ERR_ARG; }
    lc_status cs = check_search_params(sp);
    if (cs != LC_OK) return cs;
    if (!ix->trained) { set_error("search before lc_train/lc_import"); return LC_ERR_STATE; }
    if (ix->n > 0 && !ix->has_codebook) { set_error("index has no regression codebook"); return LC_ERR_STATE; }
    try {
        return lc::search(ix, q, qtype, nq, sp, nq > 0 ? ef : nullptr, ids, dists, stats, stream);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory during search");
        return LC_ERR_OOM;
    }
}

lc_status lc_search(lc_index *ix, const float *q, int64_t nq, const lc_search_params *sp,
                    int32_t *ids, float *dists, int32_t *stats, void *stream)
{
    return lc_search_ex(ix, q, LC_QUERY_F32, nq, sp, nullptr, ids, dists, stats, stream);
}

lc_status lc_autotune(lc_index *ix, const float *q, int64_t n, const int32_t *gt, const lc_tune_params *tp,
                      lc_tune_result *out)
{
    set_error("");
    if (!ix || !q || !tp || !out || n < 1) { set_error("null argument or empty sample"); return LC_ERR_ARG; }
    if (tp->k < 1 || tp->k > MAX_K || tp->ef < 1 || std::max(tp->ef, tp->k) > MAX_EF) { set_error("k or ef out of range"); return LC_ERR_ARG; }
    if (tp->max_beam < 1 || tp->max_beam > 8 || tp->reps < 1 || tp->batch < 0) {
        set_error("max_beam outside 1..8, reps < 1 or batch < 0");
        return LC_ERR_ARG;
    }
    if (!ix->trained || ix->n == 0) { set_error("autotune needs a trained, non-empty index"); return LC_ERR_STATE; }
    if (!ix->has_codebook) { set_error("index has no regression codebook"); return LC_ERR_STATE; }
    std::memset(out, 0, sizeof(*out));
    try {
        return lc::autotune(ix, q, n, gt, tp, out);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory during autotune");
        return LC_ERR_OOM;
    }
}

lc_status lc_plan_create(lc_index *ix, int64_t nq_max, const lc_search_params *sp, int qtype,
                         int per_query_ef, lc_plan **out)
{
    set_error("");
    if (!ix || !sp || !out) { set_error("null index, parameters or output"); return LC_ERR_ARG; }
    *out = nullptr;
    if (nq_max < 1 || nq_max > ((int64_t)1 << 31)) { set_error("nq_max = %lld outside 1..2^31", (long long)nq_max); return LC_ERR_ARG; }
    if (qtype != LC_QUERY_F32 && qtype != LC_QUERY_U8) { set_error("query type %d is neither LC_QUERY_F32 nor LC_QUERY_U8", qtype); return LC_ERR_ARG; }
    lc_status cs = check_search_params(sp);
    if (cs != LC_OK) return cs;
    if (!ix->trained) { set_error("plan before lc_train/lc_import"); return LC_ERR_STATE; }
    if (ix->n > 0 && !ix->has_codebook) { set_error("index has no regression codebook"); return LC_ERR_STATE; }
    try {
        return lc::plan_create(ix, nq_max, sp, qtype, per_query_ef, out);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory making a plan");
        return LC_ERR_OOM;
    }
}

lc_status lc_plan_buffers(const lc_plan *pl, void **q, int32_t **ef, int32_t **ids, float **dists, int32_t **stats)
{
    set_error("");
    if (!pl) { set_error("null plan"); return LC_ERR_ARG; }
    return lc::plan_buffers(pl, q, ef, ids, dists, stats);
}

lc_status lc_plan_run(lc_plan *pl, int64_t nq, void *stream)
{
    set_error("");
    if (!pl) { set_error("null plan"); return LC_ERR_ARG; }
    return lc::plan_run(pl, nq, stream);
}

void lc_plan_free(lc_plan *pl) { lc::plan_free(pl); }

lc_status lc_import(lc_index *ix, int64_t n, const float *R, const float *C1, const float *C2,
                    const uint8_t *codes1, const uint8_t *codes2, const uint8_t *beta,
                    const float *B, const int32_t *adj0, const int32_t *levels,
                    const int32_t *upper_adj, int32_t ep)
{
    set_error("");
    if (!ix || !R || !C1 || !C2 || !B || n < 0) { set_error("null argument"); return LC_ERR_ARG; }
    if (n > 0 && (!codes1 || !codes2 || !beta || !adj0 || !levels)) { set_error("null array"); return LC_ERR_ARG; }
    if (n > (int64_t)0x7fffffff) { set_error("too many vectors"); return LC_ERR_ARG; }
    const int d = ix->p.d, M1 = ix->p.M1, M2 = ix->p.M2, bM = ix->p.beta_M, bK = ix->p.beta_K;
    int64_t rows = 0;
    int maxl = -1;
    for (int64_t i = 0; i < n * bM; i++)
        if (beta[i] >= bK) { set_error("codeword %d of vector %lld exceeds beta_K - 1 = %d", beta[i], (long long)(i / bM), bK - 1); return LC_ERR_ARG; }
    for (int64_t i = 0; i < n; i++) {
        if (levels[i] < 0 || levels[i] > MAX_LEVEL) { set_error("level of node %lld outside 0..%d", (long long)i, MAX_LEVEL); return LC_ERR_ARG; }
        rows += levels[i];
        if (levels[i] > maxl) maxl = levels[i];
    }
    if (rows > 0 && !upper_adj) { set_error("upper_adj is NULL but some levels are positive"); return LC_ERR_ARG; }
    if (n > 0 && (ep < 0 || ep >= n || levels[ep] != maxl)) { set_error("entry point must be a node of maximal level"); return LC_ERR_ARG; }
    for (int64_t i = 0; i < n * DEG; i++)
        if (adj0[i] < -1 || adj0[i] >= n) { set_error("adj0 entry out of range at %lld", (long long)i); return LC_ERR_ARG; }
    // upper rows: node i's row for level l may only name nodes of level >= l
    {
        int64_t r = 0;
        for (int64_t i = 0; i < n; i++)
            for (int l = 1; l <= levels[i]; l++, r++)
                for (int s = 0; s < DEG; s++) {
                    int32_t v = upper_adj[r * DEG + s];
                    if (v < -1 || v >= n || (v >= 0 && levels[v] < l)) {
                        set_error("upper row of node %lld level %d names node %d", (long long)i, l, v);
                        return LC_ERR_ARG;
                    }
                }
    }
    try {
        ix->R.assign(R, R + (size_t)d * d);
        ix->C1.assign(C1, C1 + (size_t)KSUB * d);
        ix->C2.assign(C2, C2 + (size_t)KSUB * d);
        ix->B.assign(B, B + (size_t)bM * bK * (KBETA + 1));
        ix->codes1.assign(codes1, codes1 + (size_t)n * M1);
        ix->codes2.assign(codes2, codes2 + (size_t)n * M2);
        ix->beta.assign(beta, beta + (size_t)n * bM);
        ix->adj0.assign(adj0, adj0 + (size_t)n * DEG);
        ix->levels.assign(levels, levels + (size_t)n);
        ix->upper_adj.assign(upper_adj, upper_adj + (size_t)rows * DEG);
        ix->upper_off.assign((size_t)n, -1);
        int64_t r = 0;
        for (int64_t i = 0; i < n; i++) {
            if (levels[i] > 0) ix->upper_off[i] = r;
            r += levels[i];
        }
        ix->n = n;
        ix->ep = n > 0 ? ep : -1;
        ix->max_level = maxl;
        ix->trained = true;
        ix->has_codebook = true;
        ix->xh.clear();
        ix->adj0_d.clear();
        ix->upper_d.clear();
        ix->dev_dirty = true;
    } catch (const std::bad_alloc &) {
        set_error("out of host memory during import");
        return LC_ERR_OOM;
    }
    return LC_OK;
}

int64_t lc_size(const lc_index *ix) { return ix ? ix->n : 0; }

int64_t lc_upper_rows(const lc_index *ix) { return ix ? (int64_t)ix->upper_adj.size() / DEG : 0; }

lc_status lc_export(const lc_index *ix, float *R, float *C1, float *C2, uint8_t *codes1,
                    uint8_t *codes2, uint8_t *beta, float *B, int32_t *adj0, int32_t *levels,
                    int32_t *upper_adj, int32_t *ep)
{
    set_error("");
    if (!ix) { set_error("null index"); return LC_ERR_ARG; }
    if (!ix->trained) { set_error("index is not trained"); return LC_ERR_STATE; }
    auto cp = [](void *dst, const void *src, size_t bytes) { if (dst && bytes) std::memcpy(dst, src, bytes); };
    cp(R, ix->R.data(), ix->R.size() * 4);
    cp(C1, ix->C1.data(), ix->C1.size() * 4);
    cp(C2, ix->C2.data(), ix->C2.size() * 4);
    cp(codes1, ix->codes1.data(), ix->codes1.size());
    cp(codes2, ix->codes2.data(), ix->codes2.size());
    cp(beta, ix->beta.data(), ix->beta.size());
    if (ix->has_codebook) cp(B, ix->B.data(), ix->B.size() * 4);
    cp(adj0, ix->adj0.data(), ix->adj0.size() * 4);
    cp(levels, ix->levels.data(), ix->levels.size() * 4);
    cp(upper_adj, ix->upper_adj.data(), ix->upper_adj.size() * 4);
    if (ep) *ep = ix->ep;
    return LC_OK;
}

// File format (little-endian, native layouts): "LCIDX003", lc_params, int64 n, int64 upper
// rows, int32 ep, int32 max_level, int32 trained, int32 has_codebook, then R, C1, C2,
// B [beta_M][beta_K][9], codes1, codes2, beta [n][beta_M], adj0, levels, upper_adj.
static const char MAGIC[8] = {'L', 'C', 'I', 'D', 'X', '0', '0', '3'};

lc_status lc_save(const lc_index *ix, const char *path)
{
    set_error("");
    if (!ix || !path) { set_error("null argument"); return LC_ERR_ARG; }
    if (!ix->trained) { set_error("cannot save an untrained index"); return LC_ERR_STATE; }
    FILE *f = std::fopen(path, "wb");
    if (!f) { set_error("cannot open %s for writing", path); return LC_ERR_IO; }
    int64_t rows = (int64_t)ix->upper_adj.size() / DEG;
    int32_t hdr[4] = {ix->ep, ix->max_level, ix->trained ? 1 : 0, ix->has_codebook ? 1 : 0};
    bool ok = std::fwrite(MAGIC, 1, 8, f) == 8 && std::fwrite(&ix->p, sizeof(lc_params), 1, f) == 1 &&
              std::fwrite(&ix->n, 8, 1, f) == 1 && std::fwrite(&rows, 8, 1, f) == 1 &&
              std::fwrite(hdr, 4, 4, f) == 4;
    auto put = [&](const void *p, size_t bytes) { if (ok && bytes) ok = std::fwrite(p, 1, bytes, f) == bytes; };
    std::vector<float> Bz((size_t)ix->p.beta_M * ix->p.beta_K * (KBETA + 1), 0.f);
    put(ix->R.data(), ix->R.size() * 4);
    put(ix->C1.data(), ix->C1.size() * 4);
    put(ix->C2.data(), ix->C2.size() * 4);
    put(ix->has_codebook ? ix->B.data() : Bz.data(), Bz.size() * 4);
    put(ix->codes1.data(), ix->codes1.size());
    put(ix->codes2.data(), ix->codes2.size());
    put(ix->beta.data(), ix->beta.size());
    put(ix->adj0.data(), ix->adj0.size() * 4);
    put(ix->levels.data(), ix->levels.size() * 4);
    put(ix->upper_adj.data(), ix->upper_adj.size() * 4);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) { set_error("write to %s failed", path); return LC_ERR_IO; }
    return LC_OK;
}

lc_status lc_load(const char *path, lc_index **out)
{
    set_error("");
    if (!path || !out) { set_error("null argument"); return LC_ERR_ARG; }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) { set_error("cannot open %s", path); return LC_ERR_IO; }
    char magic[8];
    lc_params p;
    int64_t n = 0, rows = 0;
    int32_t hdr[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, MAGIC, 8) == 0 &&
              std::fread(&p, sizeof(p), 1, f) == 1 && std::fread(&n, 8, 1, f) == 1 &&
              std::fread(&rows, 8, 1, f) == 1 && std::fread(hdr, 4, 4, f) == 4;
    if (!ok || check_params(&p) != LC_OK || n < 0 || rows < 0 || n > (int64_t)0x7fffffff) {
        std::fclose(f);
        set_error("%s is not a valid index file", path);
        return LC_ERR_IO;
    }
    std::vector<float> R, C1, C2, B;
    std::vector<uint8_t> codes1, codes2, beta;
    std::vector<int32_t> adj0, levels, upper;
    lc_index *ix = nullptr;
    try {
        int d = p.d;
        auto get = [&](auto &vec, size_t count) {
            vec.resize(count);
            if (ok && count) ok = std::fread(vec.data(), sizeof(vec[0]), count, f) == count;
        };
        get(R, (size_t)d * d);
        get(C1, (size_t)KSUB * d);
        get(C2, (size_t)KSUB * d);
        get(B, (size_t)p.beta_M * p.beta_K * (KBETA + 1));
        get(codes1, (size_t)n * p.M1);
        get(codes2, (size_t)n * p.M2);
        get(beta, (size_t)n * p.beta_M);
        get(adj0, (size_t)n * DEG);
        get(levels, (size_t)n);
        // the upper rows are one per (node, level >= 1): a count that disagrees with the
        // levels would let the import read past the rows that were loaded
        int64_t want = 0;
        for (int32_t l : levels) want += l > 0 ? l : 0;
        if (ok && want != rows) {
            std::fclose(f);
            set_error("%s: %lld upper rows stored, the levels need %lld", path, (long long)rows, (long long)want);
            return LC_ERR_IO;
        }
        get(upper, (size_t)rows * DEG);
        if (ok && std::fgetc(f) != EOF) {
            std::fclose(f);
            set_error("%s has data after the index", path);
            return LC_ERR_IO;
        }
        ix = new lc_index();
        ix->p = p;
    } catch (const std::bad_alloc &) {
        std::fclose(f);
        delete ix;
        set_error("out of host memory loading %s", path);
        return LC_ERR_OOM;
    }
    std::fclose(f);
    if (!ok) {
        delete ix;
        set_error("%s is truncated", path);
        return LC_ERR_IO;
    }
    // validate through the import path, which also rebuilds the row offsets
    lc_status s = lc_import(ix, n, R.data(), C1.data(), C2.data(), codes1.data(), codes2.data(),
                            beta.data(), B.data(), adj0.data(), levels.data(), upper.data(), hdr[0]);
    if (s != LC_OK) {
        std::string msg = lc_last_error();
        delete ix;
        set_error("%s: %s", path, msg.c_str());
        return LC_ERR_IO;
    }
    ix->trained = hdr[2] != 0;
    ix->has_codebook = hdr[3] != 0;
    *out = ix;
    return LC_OK;
}

void lc_free(lc_index *ix)
{
    if (!ix) return;
    device_free(ix->dev);
    delete ix;
}

const char *lc_last_error(void) { return g_err; }

lc_status lc_search_walk_noalloc(lc_index *ix, const float *q, int64_t nq, int k, int ef,
                                 int32_t *ids, float *dists, int32_t *stats, void *stream)
{
    set_error("");
    if (!ix) { set_error("null index"); return LC_ERR_ARG; }
    if (nq < 0 || (nq > 0 && (!q || !ids || !dists))) { set_error("null query or output buffer"); return LC_ERR_ARG; }
    if (k < 1 || k > MAX_K) { set_error("k = %d outside 1..%d", k, MAX_K); return LC_ERR_ARG; }
    if (ef < 1) { set_error("ef must be >= 1"); return LC_ERR_ARG; }
    if (!ix->trained) { set_error("search before lc_train/lc_import"); return LC_ERR_STATE; }
    return lc::search_walk_noalloc(ix, q, nq, k, ef, ids, dists, stats, stream);
}

lc_status lc_merge_topk(const int32_t *ids, const float *dists, int S, int64_t nq, int k,
                        const int64_t *id_offsets, int32_t *ids_out, float *dists_out, void *stream)
{
    set_error("");
    if (S < 1 || S > 64 || k < 1 || nq < 0 || (int64_t)S * k > 2048) { set_error("need 1 <= S <= 64, 1 <= k, S * k <= 2048"); return LC_ERR_ARG; }
    if (nq > 0 && (!ids || !dists || !id_offsets || !ids_out || !dists_out)) { set_error("null argument"); return LC_ERR_ARG; }
    for (int s = 0; s < S; s++)
        if (id_offsets[s] < 0 || id_offsets[s] > 0x7fffffff) { set_error("id offset out of range"); return LC_ERR_ARG; }
    return lc::merge_topk(ids, dists, S, nq, k, id_offsets, ids_out, dists_out, stream);
}

lc_status lc_profile(lc_index *ix, int enable)
{
    set_error("");
    if (!ix) { set_error("null index"); return LC_ERR_ARG; }
    if (!ix->trained) { set_error("index is not trained"); return LC_ERR_STATE; }
    return lc::profile_enable(ix, enable);
}

lc_status lc_profile_read(lc_index *ix, float *walk_ms, float *refine_ms)
{
    set_error("");
    if (!ix) { set_error("null index"); return LC_ERR_ARG; }
    return lc::profile_read(ix, walk_ms, refine_ms);
}

lc_status lc_profile_phases(lc_index *ix, float *rotate_ms, float *descent_ms, float *level0_ms, float *refine_ms)
{
    set_error("");
    if (!ix) { set_error("null index"); return LC_ERR_ARG; }
    return lc::profile_phases(ix, rotate_ms, descent_ms, level0_ms, refine_ms);
}

}  // extern "C"
