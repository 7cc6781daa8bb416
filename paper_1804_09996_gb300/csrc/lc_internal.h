// Internal declarations shared by the translation units of liblc.so (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lc.h"

namespace lc {

constexpr int KSUB = 256;     // centroids per sub-quantiser (8-bit codes)
constexpr int KBETA = 8;      // neighbours in G(x)
constexpr int NBETA = 256;    // largest regression codebook (per block)
constexpr int MAX_BETA_M = 32; // most regression blocks (product codebook)
constexpr int DEG = 32;       // graph degree at every level
constexpr int MAX_LEVEL = 15; // level cap
constexpr int MAX_EF = 1024;  // largest ef' = max(efSearch, k)
constexpr int MAX_K = 256;
constexpr int MAX_SHORTLIST = 256;

void set_error(const char *fmt, ...);
lc_status check_search_params(const lc_search_params *sp);   // argument checks of lc_search

// Sub-space split: M contiguous blocks, the first (d mod M) of ceil(d/M) dimensions.
void splits(int d, int M, std::vector<int> &off, std::vector<int> &len);

// Device copy of an index (owned by lc_index, defined in lc_search.cu).
struct DeviceIndex;
void device_free(DeviceIndex *dv);

}  // namespace lc

struct lc_index {
    lc_params p{};
    bool trained = false;
    bool has_codebook = false;          // regression codebook present
    int64_t n = 0;
    std::vector<float> R;               // [d][d], y' = R y
    std::vector<float> C1, C2;          // [256][d] full-width centroids
    std::vector<uint8_t> codes1, codes2;
    std::vector<uint8_t> beta;          // [n][beta_M] codeword per block (zeros when beta_K = 1)
    std::vector<float> B;               // [beta_M][beta_K][9]
    std::vector<int32_t> adj0;          // [n][32]
    std::vector<float> adj0_d;          // build-side: distance of each row entry to its owner
    std::vector<int32_t> levels;        // [n]
    std::vector<int64_t> upper_off;     // [n], first upper row of a node or -1
    std::vector<int32_t> upper_adj;     // [rows][32]
    std::vector<float> upper_d;         // build-side distances of upper rows
    std::vector<float> xh;              // build-side decoded vectors q(x) [n][d] (rotated space)
    int32_t ep = -1;
    int max_level = -1;
    // device copy, uploaded on the first search after a change
    lc::DeviceIndex *dev = nullptr;
    bool dev_dirty = true;
};

namespace lc {
// Host build (lc_build.cpp).
lc_status build_train(lc_index *ix, const float *xt, int64_t nt);
lc_status build_add(lc_index *ix, const float *x, int64_t n);
void decode_all(const lc_index *ix, std::vector<float> &xh);
int n_threads(const lc_params &p);

// Device search (lc_search.cu).
lc_status search(lc_index *ix, const void *q, int qtype, int64_t nq, const lc_search_params *sp,
                 const int32_t *efq, int32_t *ids, float *dists, int32_t *stats, void *stream);
lc_status profile_enable(lc_index *ix, int on);
lc_status merge_topk(const int32_t *ids, const float *dists, int S, int64_t nq, int k, const int64_t *offsets,
                     int32_t *ids_out, float *dists_out, void *stream);
lc_status search_walk_noalloc(lc_index *ix, const float *q, int64_t nq, int k, int ef, int32_t *ids,
                              float *dists, int32_t *stats, void *stream);
lc_status profile_read(lc_index *ix, float *walk_ms, float *refine_ms);
lc_status profile_phases(lc_index *ix, float *rotate_ms, float *descent_ms, float *level0_ms, float *refine_ms);
// Autotuner (lc_tune.cpp).
lc_status autotune(lc_index *ix, const float *q, int64_t n, const int32_t *gt, const lc_tune_params *tp,
                   lc_tune_result *out);
// GPU-assisted build (lc_build_gpu.cu): the device copy of the index under construction serves
// the level-0 insertion searches of each batch; rows changed by a batch are re-sent.
lc_status build_gpu_begin(lc_index *ix);
// m rotated vectors xr [m][d] (host) search level 0 from ep after a greedy descent of levels
// max_level..1, keeping efc, and their neighbours are selected: select_start queues the work
// (the host may work meanwhile), select_finish waits and writes sel [m][DEG + 1] (host: ids,
// then count).  Needs build_gpu_link0_begin.
lc_status build_gpu_select_start(lc_index *ix, const float *xr, int64_t m, int efc, int32_t ep, int max_level);
lc_status build_gpu_select_finish(lc_index *ix, int64_t m, int32_t *sel);
// Re-sends level-0 rows of nodes0 [n0] and upper rows (indexes into upper_adj) rows_up [nu].
lc_status build_gpu_rows(lc_index *ix, const int32_t *nodes0, int64_t n0, const int64_t *rows_up, int64_t nu);
void build_gpu_end(lc_index *ix);
// Level-0 linking of a batch on the device (lc_build_gpu.cu).  link0_begin uploads the decoded
// vectors (ix->xh) and the level-0 row distances (ix->adj0_d) of the whole index.  link0 takes
// the level-0 selections of the batch's members first .. first + b - 1 (sel0 [b][DEG + 1]:
// ids, then count) and the batch's level-0 back-links grouped by target (targets [G], group
// g's sources src[starts[g] .. starts[g + 1]) in increasing id), writes the members' own rows
// and applies the back-links on the device copy exactly as the host build does, then copies
// the ids of every row it wrote back into ix->adj0; link0_end copies the level-0 row distances
// back into ix->adj0_d.
lc_status build_gpu_link0_begin(lc_index *ix);
lc_status build_gpu_link0(lc_index *ix, int64_t first, int64_t b, const int32_t *sel0, const int32_t *targets,
                          const int32_t *starts, int64_t G, const int32_t *src);
lc_status build_gpu_link0_end(lc_index *ix);
// Codeword assignment of vectors [first, first + n) (rotated xr [n][d], host) on the device,
// after the graph is final; writes ix->beta exactly as the host assignment would.
lc_status build_gpu_assign(lc_index *ix, const float *xr, int64_t first, int64_t n);
// Regression-codebook training on the device (lc_build_gpu.cu), in the host build's double
// arithmetic.  em_begin uploads the k-means points X [n][dim] (dim <= 16) and the samples'
// normal equations ne55 [n][55] (A packed upper triangle 45, b 9, ||x||^2); em_nearest writes
// each point's nearest centre of C [K][dim] (cn [K]: squared norms) and its squared distance;
// em_assign writes each sample's argmin codeword of B [K][9].  NULL / false on a CUDA failure.
struct EmDev;
EmDev *em_begin(const double *X, int64_t n, int dim, const double *ne55);
bool em_nearest(EmDev *em, const double *C, const double *cn, int K, int32_t *as, double *dm);
bool em_assign(EmDev *em, const double *B, int K, int32_t *as);
void em_free(EmDev *em);
// Rotation and two-level encoding of x [n][d] (host) on the device, with the host build's
// arithmetic: xr [n][d], codes c1 [n][M1], c2 [n][M2] (host).
lc_status build_gpu_encode(lc_index *ix, const float *x, int64_t n, float *xr, uint8_t *c1, uint8_t *c2);
// Captured searches (lc_plan_*), lc_search.cu.
lc_status plan_create(lc_index *ix, int64_t nq_max, const lc_search_params *sp, int qtype, int per_query_ef,
                      lc_plan **out);
lc_status plan_buffers(const lc_plan *pl, void **q, int32_t **ef, int32_t **ids, float **dists, int32_t **stats);
lc_status plan_run(lc_plan *pl, int64_t nq, void *stream);
void plan_free(lc_plan *pl);
}  // namespace lc
