// Host-side view of the device index and of one search's launch plan and scratch, shared by
// the search (lc_search.cu), the GPU-assisted build (lc_build_gpu.cu) and the request server
// (lc_serve.cpp).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lc_internal.h"

namespace lc {

struct DeviceIndex {
    int device = -1;
    int64_t n = 0;
    int d = 0, M1 = 0, M2 = 0, max_level = 0;
    int32_t ep = -1;
    float *Rt = nullptr;          // [d][d], Rt[u*d + t] = R[t][u]
    float *C1 = nullptr, *C2 = nullptr, *B = nullptr;
    float *C1w = nullptr;         // C1 in the walk's shared-memory layout (FP32)
    void *C1h = nullptr;          // the same rounded to FP16 (device __half), for the FP16 mode
    void *C2h = nullptr;          // C2 rounded to FP16 [256][d] (full-decode walk in FP16)
    uint8_t *codes1 = nullptr, *codes2b = nullptr;   // codes2b: residual codes padded to M2P bytes, codeword id last
    int M2P = 0;
    int bM = 1, bK = 256;         // regression blocks and codewords per block (B: [bM][bK][9])
    int32_t *adj0 = nullptr, *upper_off = nullptr, *upper_adj = nullptr;
    // scratch of lc_search, grown on demand
    float *yq = nullptr; size_t yq_cap = 0;
    int32_t *shortlist = nullptr; size_t sl_cap = 0;
    int32_t *spill = nullptr; size_t spill_cap = 0;
    int32_t *ord = nullptr; size_t ord_cap = 0;       // ordered search: 4 words per query
    uint16_t *tab = nullptr; size_t tab_cap = 0;      // table form: FP16 ADC tables [nq][256][32]
    int32_t *status = nullptr;
    unsigned long long *counter = nullptr;
    // staging for host-pointer calls
    float *q_st = nullptr; size_t q_cap = 0;
    int32_t *ef_st = nullptr; size_t ef_cap = 0;
    int32_t *ids_st = nullptr; float *d_st = nullptr; int32_t *s_st = nullptr; size_t out_cap = 0;
    // profiling
    bool profile = false;
    // profiled search: before the rotation, after the level-0 walk, after the refinement,
    // after the rotation, before the level-0 walk (after the descent and the sort)
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_valid = false, has_refine = false;
    int num_sms = 0;
    uint64_t gen = 0;             // changes with every upload (plans check it)
    // GPU-assisted build: batch vectors, results and re-sent rows
    float *b_yq = nullptr; size_t b_yq_cap = 0;
    int32_t *b_ids = nullptr; size_t b_ids_cap = 0;
    float *b_d = nullptr; size_t b_d_cap = 0;
    int32_t *b_rows = nullptr; size_t b_rows_cap = 0;
    int64_t *b_idx = nullptr; size_t b_idx_cap = 0;
    int32_t *b_sel = nullptr; size_t b_sel_cap = 0;
    struct LinkDev *lk = nullptr;  // level-0 linking of the GPU-assisted build (lc_build_gpu.cu)
};

// Frees the level-0 linking state of the GPU-assisted build (no-op without one).
void link0_free(DeviceIndex *dv);

inline void cfree(void *p) { if (p) cudaFree(p); }

// dst = a fresh device copy of src (at least 16 bytes allocated)
template <class T>
inline bool dupload(T *&dst, const std::vector<T> &src)
{
    cfree(dst);
    dst = nullptr;
    size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
    if (cudaMalloc(&dst, bytes) != cudaSuccess) return false;
    if (!src.empty() && cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    return true;
}

// p holds at least need elements (reallocated, contents dropped, when it is smaller)
template <class T>
inline bool grow(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return true;
    cfree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) return false;
    cap = need;
    return true;
}

// Launch configuration of one search and the scratch it needs.
struct SearchPlan {
    int k = 0, efp = 0, R = 0, beam = 1, tcap = 0, hash_log = 0, spill_log = 0, variant = 0;
    bool refine = false;
    bool half = false;                   // FP16 level-1 codebook in the walk
    bool full = false;                   // the walk scores the full two-level decode
    int wpc = 0, grid = 0;               // walk: warps per CTA, CTAs
    size_t per_warp = 0, smem = 0;
    int rw = 0, rgrid = 0;               // refine: warps per CTA, CTAs
    int qgrid = 0;                       // rotation: CTAs
    size_t qsm = 0;                      // rotation: shared memory
    size_t rsm = 0;
    bool rboth = false;                  // both codebooks in shared memory
    bool ordered = false;                // two walk launches, level 0 in decreasing entry distance
    bool tab = false;                    // table form: table_kernel, then the walk's table instantiation
    size_t tab_elems = 0;                // FP16 table entries of the batch
    int dwpc = 0, dgrid = 0;             // ordered search: the descent launch's warps per CTA, CTAs
    size_t dsmem = 0;
    size_t yq_elems = 0, sl_elems = 0, spill_elems = 0, ord_elems = 0;
};

// Device scratch of one search in flight.
struct SearchScratch {
    float *yq = nullptr;                 // [nq][d] rotated queries
    int32_t *shortlist = nullptr;        // [nq][R] (refinement only)
    int32_t *spill = nullptr;            // [grid * wpc][2^spill_log]
    uint16_t *tab = nullptr;             // table form: [nq][256][32] FP16
    int32_t *ord = nullptr;              // ordered search: entry node, upper evaluations, queue
                                         // order (int32) and entry distance (float), [nq] each
    int32_t *status = nullptr;           // 1 word
    unsigned long long *counter = nullptr;
};

lc_status upload(lc_index *ix);

// allow_order: the caller provides the ordered search's scratch (lc_search / lc_search_ex do;
// plans, served requests and the build's searches walk in query order).
lc_status plan_search(const DeviceIndex *dv, int64_t nq, const lc_search_params *sp, SearchPlan *pl,
                      bool allow_order = false);
// Queues the walk (and refinement) on `st`; q, ids, dists, stats are device pointers.
// q8 (uint8 queries [nq][d], replacing q) and efq (per-query efSearch [nq]) are optional
// device pointers; rotated: sc.yq already holds y' (no rotation launch, q unused).
lc_status run_search(DeviceIndex *dv, const SearchPlan &pl, const float *q, int64_t nq, int32_t *ids,
                     float *dists, int32_t *stats, const SearchScratch &sc, cudaStream_t st, bool profile,
                     const uint8_t *q8 = nullptr, const int32_t *efq = nullptr, bool rotated = false);

}  // namespace lc
