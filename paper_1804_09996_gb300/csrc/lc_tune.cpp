// Autotuner of the search (lc_autotune): picks the beam width, codebook precision and
// efSearch that reach a recall target at the least time, then the launch shape (queries in
// flight per block, visited-table size) that runs those parameters fastest.  The first stage
// changes results and is judged by 1-recall@1 on the caller's sample; the second cannot
// change results (the visited set is exact whatever its table size, and the launch shape only
// changes which warp runs which query).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "lc_internal.h"

namespace lc {
namespace {

struct Sample {
    float *q = nullptr;
    int32_t *ids = nullptr;
    float *dists = nullptr;
    int64_t n = 0;        // distinct sample queries (recall)
    int64_t nb = 0;       // queries per timed search (the sample repeated)
    int k = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Sample()
    {
        if (q) cudaFree(q);
        if (ids) cudaFree(ids);
        if (dists) cudaFree(dists);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
};

struct Measured {
    lc_status status = LC_OK;
    float ms = INFINITY, recall = 0.f;
    std::vector<int32_t> top1;
};

// Median time of `reps` searches of the sample (after one untimed run) and the top-1 ids.
Measured measure(lc_index *ix, Sample &s, const lc_search_params &sp, int reps, const std::vector<int32_t> *ref)
{
    Measured m;
    m.status = search(ix, s.q, LC_QUERY_F32, s.nb, &sp, nullptr, s.ids, s.dists, nullptr, s.st);
    if (m.status != LC_OK) return m;
    std::vector<float> t;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(s.e0, s.st);
        m.status = search(ix, s.q, LC_QUERY_F32, s.nb, &sp, nullptr, s.ids, s.dists, nullptr, s.st);
        cudaEventRecord(s.e1, s.st);
        if (m.status != LC_OK) return m;
        if (cudaEventSynchronize(s.e1) != cudaSuccess) {
            set_error("timing the search failed: %s", cudaGetErrorString(cudaGetLastError()));
            m.status = LC_ERR_CUDA;
            return m;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s.e0, s.e1);
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    m.ms = t[t.size() / 2];
    std::vector<int32_t> all((size_t)s.n * s.k);
    if (cudaMemcpy(all.data(), s.ids, all.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("reading the sample's results failed");
        m.status = LC_ERR_CUDA;
        return m;
    }
    m.top1.resize(s.n);
    for (int64_t i = 0; i < s.n; i++) m.top1[i] = all[(size_t)i * s.k];
    if (ref) {
        int64_t hit = 0;
        for (int64_t i = 0; i < s.n; i++) hit += m.top1[i] == (*ref)[i];
        m.recall = (float)hit / (float)s.n;
    }
    return m;
}

}  // namespace

lc_status autotune(lc_index *ix, const float *q, int64_t n, const int32_t *gt, const lc_tune_params *tp,
                   lc_tune_result *out)
{
    const int d = ix->p.d;
    Sample s;
    s.n = n;
    s.nb = std::max<int64_t>(n, tp->batch);
    s.k = tp->k;
    if (cudaMalloc(&s.q, (size_t)s.nb * d * 4) != cudaSuccess || cudaMalloc(&s.ids, (size_t)s.nb * tp->k * 4) != cudaSuccess ||
        cudaMalloc(&s.dists, (size_t)s.nb * tp->k * 4) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s.e0) != cudaSuccess || cudaEventCreate(&s.e1) != cudaSuccess) {
        set_error("autotune: device allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return LC_ERR_OOM;
    }
    for (int64_t a = 0; a < s.nb; a += n) {
        const int64_t c = std::min(n, s.nb - a);
        if (cudaMemcpy(s.q + a * d, q, (size_t)c * d * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("autotune: sample upload failed");
            return LC_ERR_CUDA;
        }
    }
    const int reps = std::max(1, tp->reps);
    // reference top-1: the caller's exact neighbours, or the plain search at 4x efSearch
    std::vector<int32_t> ref;
    lc_search_params base;
    lc_default_search_params(&base, tp->k, tp->ef);
    if (gt) {
        ref.assign(gt, gt + n);
    } else {
        lc_search_params wide = base;
        wide.ef = std::min(MAX_EF, 4 * tp->ef);
        Measured w = measure(ix, s, wide, 1, nullptr);
        if (w.status != LC_OK) return w.status;
        ref = w.top1;
    }
    Measured b = measure(ix, s, base, reps, &ref);
    if (b.status != LC_OK) return b.status;
    out->target = b.recall;
    out->base_ms = b.ms;
    out->sp = base;
    out->ms = b.ms;
    out->recall = b.recall;
    out->tried = 1;
    // stage 1: per (beam, precision), the smallest efSearch on a ladder around ef that reaches
    // the target; keep the fastest
    const int ladder_num[] = {2, 3, 4, 5, 6, 7, 8, 10, 12, 16};   // eighths of ef
    const int max_beam = std::min(8, std::max(1, tp->max_beam));
    for (int beam = 1; beam <= max_beam; beam *= 2) {
        for (int prec = 0; prec <= (tp->allow_fp16 ? 1 : 0); prec++) {
            int last = -1;
            for (int num : ladder_num) {
                int ef = std::max(1, (tp->ef * num + 4) / 8);
                if (ef == last) continue;
                last = ef;
                lc_search_params sp = base;
                sp.ef = ef;
                sp.lut_prec = prec ? LC_LUT_FP16 : LC_LUT_FP32;
                sp.mode = beam > 1 ? LC_MODE_BATCHED : LC_MODE_PLAIN;
                sp.beam = beam;
                Measured m = measure(ix, s, sp, reps, &ref);
                out->tried++;
                if (m.status == LC_ERR_CAPACITY) break;           // wider searches cannot fit either
                if (m.status != LC_OK) return m.status;
                if (m.recall >= out->target) {
                    if (m.ms < out->ms) { out->sp = sp; out->ms = m.ms; out->recall = m.recall; }
                    break;
                }
            }
        }
    }
    // stage 2: launch shape for the chosen parameters (results unchanged)
    const lc_search_params chosen = out->sp;
    for (int vlog : {0, 10, 11, 12}) {
        for (int warps : {0, 4, 8, 12}) {
            if (vlog == 0 && warps == 0) continue;
            lc_search_params sp = chosen;
            sp.visited_log = vlog;
            sp.warps = warps;
            Measured m = measure(ix, s, sp, reps, &ref);
            out->tried++;
            if (m.status == LC_ERR_CAPACITY) continue;
            if (m.status != LC_OK) return m.status;
            if (m.ms < out->ms) { out->sp = sp; out->ms = m.ms; out->recall = m.recall; }
        }
    }
    return LC_OK;
}

}  // namespace lc
