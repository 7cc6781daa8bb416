/*
 * lc.h - C ABI of the GB300 Link-and-Code library (liblc.so).
 *
 * Link and Code (Douze, Sablayrolles, Jegou, CVPR 2018) indexes vectors with a
 * two-level product-quantisation code and an HNSW-style neighbour graph, and refines
 * the distance estimate of short-listed candidates by regression from their graph
 * neighbours' codes.  This library builds such an index on the host and answers k-NN
 * queries on the GPU.
 *
 * Conventions (every entry point):
 *   - Returns lc_status and never aborts.  Arguments are checked before any device work;
 *     on error nothing is written to the caller's outputs and lc_last_error() gives a
 *     message (per calling thread).
 *   - The library owns the index and every device allocation it makes.  The caller owns
 *     its own buffers; the library never frees or retains them past the call (for an
 *     asynchronous search: past completion of the work queued on the given stream).
 *   - Row-major arrays: [n][d] means n rows of d contiguous elements.
 *   - Ordering of results is by (distance, id), smaller id first on equal distances.
 *   - An index is not safe for concurrent mutation; concurrent lc_search calls on one
 *     index from several host threads are not supported (serialise them).
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_index lc_index;   /* opaque; created by lc_create/lc_load, freed by lc_free */

typedef enum {
    LC_OK = 0,
    LC_ERR_ARG = 1,       /* invalid argument (null pointer, size, parameter out of range) */
    LC_ERR_OOM = 2,       /* host or device allocation failed */
    LC_ERR_STATE = 3,     /* call not valid in the index's current state */
    LC_ERR_CUDA = 4,      /* a CUDA runtime call failed (no device, launch error, ...) */
    LC_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    LC_ERR_BUDGET = 6,    /* a request can never fit the serving memory budget */
    LC_ERR_IO = 7,        /* file could not be read or written, or has a bad format */
    LC_ERR_CAPACITY = 8   /* a per-query work table overflowed (search too wide) */
} lc_status;

/* Index parameters.  Section 4.1: HNSW with degree 32 at the upper levels and a size ratio
 * of 30 between levels; Section 3.3/4.1: two-level codec, (O)PQ level 1 and a residual PQ
 * level 2, 8 bits per sub-quantiser; Section 4.3: regression over self + k = 8 neighbours
 * with a 256-entry codebook; Section 5: codebook trained on 250k vectors, 10 iterations. */
typedef struct {
    int d;                 /* vector dimension, 1..256 */
    int M1;                /* level-1 sub-quantisers: 16, 32 or 64 (bytes per vector) */
    int M2;                /* level-2 (residual) sub-quantisers, 1..256, M2 <= d */
    int use_opq;           /* 1: learn an OPQ rotation for level 1; 0: identity */
    int deg;               /* level-0 degree; must be 32 */
    int deg_upper;         /* upper-level degree; must be 32 */
    int level_ratio;       /* size ratio between consecutive levels (30) */
    int ef_construction;   /* beam width of the insertion search (40) */
    int beta_train_n;      /* vectors used to train the regression codebook (250000) */
    int beta_iters;        /* EM iterations of the codebook training (10) */
    int kmeans_iters;      /* Lloyd iterations of each PQ k-means (25) */
    int opq_iters;         /* alternations of the OPQ training (10) */
    int batch_max;         /* largest insertion batch (4096); 1 = sequential insertion */
    int n_threads;         /* host threads for train/add; 0 = all hardware threads */
    uint64_t seed;         /* seeds every random choice of the build */
    int beta_M;            /* regression blocks (Section 4.3, product codebook): the coordinates
                              split into beta_M contiguous blocks (the PQ split rule), each with
                              its own codebook; 1..min(32, d), default 1 */
    int beta_K;            /* codewords per block, 1..256 (256).  > 1: codeword 0 of every
                              block is e0 and beta_M bytes are stored per vector; 1: the 0-byte
                              refinement of Section 4.2 (one least-squares weight vector per
                              block, shared by all vectors, nothing stored per vector) */
    int build_gpu;         /* 1: lc_add runs the level-0 insertion searches of each batch on the
                              current GPU (the batch searches the graph as it stood at the batch
                              start, Section 5.1, all its level-0 members at once, with the
                              exact-to-decoded distance of the full-decode walk); neighbour
                              selection, links and the few nodes of higher level stay on the
                              host.  0 (default): everything on the host */
} lc_params;

/* Fills *p with the defaults above for dimension d and code sizes M1, M2. */
void lc_default_params(lc_params *p, int d, int M1, int M2);

/* Search modes.  PLAIN: the best-first walk of Section 2, one expansion at a time.
 * BATCHED: each step expands the `beam` best unexpanded members of the result set together
 * and merges all their new neighbours at once (a node shared by two of their rows is scored
 * once); a deterministic variant with more work in flight per query, compared with PLAIN at
 * equal recall (beam = 1 would be PLAIN). */
enum { LC_MODE_PLAIN = 0, LC_MODE_BATCHED = 1 };
/* Precision of the level-1 codebook the walk scores with (the ADC terms).  FP32: exact FP32
 * terms.  FP16: the codebook rounded to FP16 (nearest even) and held at half the shared
 * memory, so more queries are in flight per SM; arithmetic stays FP32, and the re-rank always
 * uses the FP32 codebooks.  TABLE: per-query ADC tables (Section 4.1): a tensor-core kernel
 * builds, for the whole batch, every query's table of ||y'_j - C1_j[c]||^2 over sub-spaces j
 * and centroids c (y' and C1 rounded to FP16, FP32 accumulation, entries stored in FP16, 16 KB
 * per query), and the walk and the upper-level descent add table entries; for 32 level-1
 * sub-spaces at d = 96 and the level-1 walk (LC_ERR_ARG otherwise), in every search call
 * (lc_search, lc_search_ex, plans, the server).  FP16 and TABLE change distances at FP16
 * precision. */
enum { LC_LUT_FP32 = 0, LC_LUT_FP16 = 1, LC_LUT_TABLE = 2 };

/* Search parameters (Section 2 search, Section 4.1 two-stage strategy). */
typedef struct {
    int k;           /* neighbours returned per query, 1..256 */
    int ef;          /* efSearch: size of the result set W of the walk; ef' = max(ef, k) <= 1024 */
    int shortlist;   /* 0: refine max(k, 10) candidates (Section 5.1 refines at most 10);
                        > 0: refine max(shortlist, k) (at most 256); < 0: no refinement,
                        return the walk's own top-k by ADC distance */
    int lut_prec;    /* LC_LUT_FP32, LC_LUT_FP16 or LC_LUT_TABLE */
    int mode;        /* LC_MODE_PLAIN or LC_MODE_BATCHED */
    int visited_log; /* 0: automatic; 10..14: the per-query visited table in shared memory has
                        2^visited_log entries (ids beyond three quarters of it go to a table
                        in global memory, see spill_log) */
    int beam;        /* LC_MODE_BATCHED: expansions per step, 2..8 (ignored in PLAIN mode) */
    int max_dist;    /* search-time cap T (Section 3.1): 0 = none; > 0: the level-0 search stops
                        before an expansion once T distances have been computed there */
    int warps;       /* walk queries in flight per thread block: 0 = as many as fit in shared
                        memory (at most 16); 1..16 = at most that many.  Results do not depend
                        on it (a launch-shape knob for the autotuner) */
    int walk_full;   /* 0: the walk scores the level-1 code by ADC (the default reading of
                        Section 4.1); 1: it scores the full two-level decode q = c1 + c2 (each
                        coordinate's level-1 plus level-2 centroid; reads M1 + M2P code bytes
                        per node).  With LC_LUT_FP16 both codebooks are rounded, which needs a
                        uniform level-1 split (M1 = 16 or 32 at d = 96, M1 = 64 at d = 128) */
    int order;       /* order in which the walk takes the queries (lc_search, lc_search_ex and the
                        server's launches; plans always use query order).  LC_ORDER_AUTO (0):
                        ordered once the batch has at least twice as many queries as the GPU
                        walks at once; LC_ORDER_NEVER: query order; LC_ORDER_ALWAYS: ordered.
                        Ordered: a first launch runs every query's upper-level descent, the
                        queries are sorted by decreasing distance to the node where it enters
                        level 0 (those tend to walk longest), and the level-0 searches run in
                        that order, so the batch does not end on a few long walks.  Results do
                        not depend on it */
    int spill_log;   /* the per-query visited table in global memory (one per query in flight,
                        taking the ids once the shared table is three quarters full):
                        0 = automatic, 2^13 .. 2^16 entries as max(ef, k) grows (64 entries per
                        result-set slot); 8..16: 2^spill_log entries.  A query that would fill it beyond
                        half fails: LC_ERR_CAPACITY (host pointers) or n_dist = -1 and ids -1
                        (device pointers), the other queries of the batch are unaffected */
} lc_search_params;

enum { LC_ORDER_AUTO = 0, LC_ORDER_NEVER = 1, LC_ORDER_ALWAYS = 2 };

void lc_default_search_params(lc_search_params *p, int k, int ef);

/* Creates an empty index.  *out receives the handle.  Errors: LC_ERR_ARG (bad params),
 * LC_ERR_OOM. */
lc_status lc_create(const lc_params *params, lc_index **out);

/* Trains the codec on nt host vectors xt [nt][d] (float32): the OPQ rotation (if enabled)
 * and the level-1 PQ (Section 3.3, 5.1 "systematically perform a rotation"), then the
 * residual level-2 PQ on x' - c1(x') (Section 3.3, 4.1).  Host computation.  Errors:
 * LC_ERR_ARG (nt < 256 or null), LC_ERR_STATE (already trained). */
lc_status lc_train(lc_index *ix, const float *xt, int64_t nt);

/* Adds n host vectors x [n][d] (float32), ids continuing from the current count.  Encodes
 * them with the two-level codec, inserts them into the HNSW graph by batches (Section 2,
 * 5.1; the inserted vector is compared exactly with the decoded indexed vectors, Section
 * 4.1), trains the regression codebook on the first call (Section 4.3, EM from a k-means
 * initialisation), and assigns each new vector the codeword minimising
 * ||x - beta^T G(x)||^2 (Section 4.3).  Host computation; with params.build_gpu = 1 the
 * encoding, the level-0 insertion searches, the neighbour selection and the codeword
 * assignment run on the current GPU (same results as the host build up to FP32 near-ties).
 * Errors: LC_ERR_ARG, LC_ERR_STATE (not trained), LC_ERR_OOM, LC_ERR_CUDA (build_gpu = 1
 * without a usable device, checked before the index is touched, or a device failure). */
lc_status lc_add(lc_index *ix, const float *x, int64_t n);

/* lc_add for uint8 vectors x [n][d] (integer-valued descriptors, Section 5.1), converted
 * exactly to float32 on the host first (n * d * 4 bytes of host memory for the call). */
lc_status lc_add_u8(lc_index *ix, const uint8_t *x, int64_t n);

/* k-NN search for nq queries q [nq][d] (float32): ADC walk over the nested graphs, then
 * re-rank of the shortlist with the refined reconstruction (Section 4.1, 4.3).
 * Outputs: ids [nq][k] (int32, -1 where fewer than k results), dists [nq][k] (float32
 * squared L2 to the refined reconstruction, or the ADC distance when shortlist < 0; +inf
 * with id -1), stats [nq][3] (int32: distinct nodes scored at level 0, level-0
 * expansions, evaluations on the upper levels; may be NULL).
 * Pointers may all be host memory or all device memory of the current device (checked with
 * cudaPointerGetAttributes; another GPU's memory is LC_ERR_ARG).  Device pointers: the work is queued on `stream` (a
 * cudaStream_t, NULL = the default stream) and the call returns without waiting.  Host
 * pointers: the call copies through the device and returns when the results are written.
 * The index is uploaded to the current device on the first search.
 * Errors: LC_ERR_ARG, LC_ERR_STATE (empty codec), LC_ERR_CUDA, LC_ERR_OOM,
 * LC_ERR_CAPACITY (host pointers only: some query's visited set overflowed; device
 * pointers report it as stats n_dist = -1 for that query). */
lc_status lc_search(lc_index *ix, const float *q, int64_t nq, const lc_search_params *sp,
                    int32_t *ids, float *dists, int32_t *stats, void *stream);

/* Query element types of lc_search_ex. */
enum { LC_QUERY_F32 = 0, LC_QUERY_U8 = 1 };

/* lc_search with two generalisations (the search itself is the one of Section 2, 4.1, 4.3):
 * - qtype LC_QUERY_U8: q points to uint8 queries [nq][d] (integer-valued descriptors such as
 *   SIFT, Section 5.1), converted exactly to float32 on the device; LC_QUERY_F32: float32
 *   [nq][d] as in lc_search.
 * - ef non-NULL: per-query efSearch [nq] (int32, same memory kind as q).  Query i walks with
 *   ef' = max(ef[i], k); sp->ef is the bound every ef[i] must respect (it sizes the per-query
 *   state, so a small bound keeps more queries in flight).  Host arrays are checked
 *   (LC_ERR_ARG for ef[i] outside 1..sp->ef); device arrays are clamped into 1..sp->ef.
 *   Each query's result equals that of lc_search with sp->ef = ef[i].
 * Everything else (pointer kinds, outputs, errors, stream semantics) is as lc_search;
 * lc_search(...) is lc_search_ex with LC_QUERY_F32 and ef = NULL. */
lc_status lc_search_ex(lc_index *ix, const void *q, int qtype, int64_t nq, const lc_search_params *sp,
                       const int32_t *ef, int32_t *ids, float *dists, int32_t *stats, void *stream);

/* Replaces the index's content with caller-provided host arrays (copied): rotation R
 * [d][d] (y' = R y), level-1 and level-2 centroids C1, C2 [256][d] (full width: row c holds
 * centroid c of every sub-space in that sub-space's coordinates), codes1 [n][M1],
 * codes2 [n][M2], beta [n][beta_M] (codeword id per regression block, each < beta_K; all
 * zero when beta_K = 1), regression codebooks B [beta_M][beta_K][9] (Section 4.3; with the
 * default beta_M = 1, beta_K = 256: beta [n] and B [256][9]), level-0
 * adjacency adj0 [n][32] (-1 padded, first 8 entries = the neighbours of G(x)), levels [n],
 * upper_adj [sum(levels)][32] (node i with level L >= 1 owns L consecutive rows, levels 1..L,
 * in id order), entry point ep (a node of maximal level).  Sub-space split: M blocks of
 * contiguous dimensions, the first (d mod M) of size ceil(d/M).  The index becomes trained
 * and searchable.  Errors: LC_ERR_ARG (shapes, ids or codewords out of range), LC_ERR_OOM. */
lc_status lc_import(lc_index *ix, int64_t n, const float *R, const float *C1, const float *C2,
                    const uint8_t *codes1, const uint8_t *codes2, const uint8_t *beta,
                    const float *B, const int32_t *adj0, const int32_t *levels,
                    const int32_t *upper_adj, int32_t ep);

/* Number of indexed vectors (0 for a null handle). */
int64_t lc_size(const lc_index *ix);

/* Rows of upper adjacency (sum of node levels). */
int64_t lc_upper_rows(const lc_index *ix);

/* Copies the index arrays out to caller host buffers with the layouts of lc_import (any
 * pointer may be NULL to skip it).  *ep receives the entry point.  Errors: LC_ERR_STATE. */
lc_status lc_export(const lc_index *ix, float *R, float *C1, float *C2, uint8_t *codes1,
                    uint8_t *codes2, uint8_t *beta, float *B, int32_t *adj0, int32_t *levels,
                    int32_t *upper_adj, int32_t *ep);

/* Writes the index to a file (versioned binary format) / reads one into a new handle.
 * lc_load checks the file as lc_import checks its arguments, and also that the stored count
 * of upper rows equals the sum of the levels and that nothing follows the last array; any
 * failure leaves *out NULL.  Errors: LC_ERR_IO (unreadable, truncated, inconsistent or
 * invalid file), LC_ERR_STATE (save of an untrained index), LC_ERR_OOM. */
lc_status lc_save(const lc_index *ix, const char *path);
lc_status lc_load(const char *path, lc_index **out);

/* The level-0 walk of lc_search without refinement (as lc_search with shortlist < 0:
 * outputs the walk's own top-k by ADC distance, same layouts), for callers that cannot let
 * the library allocate device memory while they serve.  cudaMalloc and cudaFree may
 * synchronise the whole device and take unbounded time, which a latency-bound request loop
 * cannot afford, and an application that manages device memory through its own pool or a
 * fixed budget cannot have memory taken behind its back.  This call allocates nothing: its
 * scratch is a file-scope device array of 64 MiB + 256 B in liblc.so (held on every GPU that
 * loads the library until the process exits), looked up once per device on the call's first
 * use there, so make that first call before any stream capture.  Each query in flight gets
 * the visited tables lc_search gives it at the same efSearch, so results (overflows
 * included) are those of lc_search; the array bounds the queries in flight (2,048 up to
 * max(ef, k) = 128, 1,024 up to 256).  The paper has no counterpart; it is an operational
 * variant of the search above.
 * Requirements: q, ids, dists (and stats, may be NULL) are device pointers of the current
 * device; the index is already resident on the current device (an earlier lc_search uploads
 * it), else LC_ERR_STATE; max(ef, k) <= 256, else LC_ERR_ARG.  Work is queued on `stream` and
 * the call returns without waiting.  Every call shares the one scratch array, so calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must be serialised by
 * the caller.  A query whose visited set overflows its table reports n_dist = -1 in stats and
 * ids -1 (as lc_search with device pointers).  Errors: LC_ERR_ARG, LC_ERR_STATE, LC_ERR_CUDA,
 * LC_ERR_CAPACITY. */
lc_status lc_search_walk_noalloc(lc_index *ix, const float *q, int64_t nq, int k, int ef,
                                 int32_t *ids, float *dists, int32_t *stats, void *stream);

/* Merges per-shard search results into global top-k lists.  A database split into S shards of
 * contiguous id ranges, each with its own index, is searched by running every query against
 * every shard; this call merges the S result lists of each query by (distance, global id),
 * global id = shard-local id + id_offsets[s] (-1 entries are padding).  The paper searches one
 * index; sharding is this library's way to hold larger databases or use several GPUs.
 * ids, dists: device arrays [S][nq][k] (the shards' outputs stacked); id_offsets: host [S];
 * ids_out, dists_out: device [nq][k].  Queued on `stream`.  Requires S <= 64, S * k <= 2048.
 * Errors: LC_ERR_ARG, LC_ERR_CUDA. */
lc_status lc_merge_topk(const int32_t *ids, const float *dists, int S, int64_t nq, int k,
                        const int64_t *id_offsets, int32_t *ids_out, float *dists_out, void *stream);

/* ---- Serving: continuous batching of requests on one GPU (the paper has no serving
 * component; this is the library's own).  The index stays resident; each request is a batch of
 * 1..max_request host queries with its own k, efSearch, shortlist and mode.  Requests wait in
 * arrival order; whenever one of the max_inflight launch slots is free, the oldest waiting
 * request starts together with every later waiting request of the same parameters up to
 * efSearch (same k, shortlist, mode, beam, codebook precision, caps and table sizes, and
 * max(ef, k) in the same power-of-two class), up to 16,384 queries (or max_request): their
 * queries run as one launch in which each query walks with its own request's efSearch.  Under
 * light load a request starts alone as soon as it arrives and overlaps with those already on
 * the GPU; under heavy load the requests that queued while the slots were busy run as a few
 * large launches.  Each launch's device state (queries, results, search scratch) is
 * sub-allocated from one arena of device_budget_bytes created at open; a merge is cut short
 * where the arena has no room.  Results are exactly those of lc_search with each request's
 * parameters.  A server is driven by one host thread: submit, poll and close from the same
 * thread. */
typedef struct lc_server lc_server;

/* Completion callback, invoked from lc_serve_poll or lc_serve_close on the calling thread.
 * status LC_OK: ids/dists hold [nq][k] results (as lc_search), valid only during the call.
 * Otherwise ids/dists must not be read: LC_ERR_CAPACITY (a query's visited set overflowed),
 * LC_ERR_CUDA, or LC_ERR_STATE (cancelled by lc_serve_close before it started). */
typedef void (*lc_request_cb)(void *user, uint64_t req_id, lc_status status, const int32_t *ids,
                              const float *dists, int32_t nq, int32_t k);

/* Opens a server on the index's device (uploads the index if needed).  Errors: LC_ERR_ARG,
 * LC_ERR_STATE (untrained or empty index), LC_ERR_OOM (budget or staging allocation),
 * LC_ERR_CUDA. */
lc_status lc_serve_open(lc_index *ix, size_t device_budget_bytes, int max_inflight, int max_request,
                        lc_server **out);

/* Queues a request (host queries q [nq][d], copied before returning) and starts it if it can
 * start now; never waits for the device.  *req_id (may be NULL) receives its id (increasing).
 * Errors: LC_ERR_ARG (as lc_search), LC_ERR_BUDGET (more than max_request queries, or more
 * device state than the whole budget: it could never be admitted), LC_ERR_CAPACITY, LC_ERR_OOM. */
lc_status lc_serve_submit(lc_server *s, const float *q, int32_t nq, const lc_search_params *sp,
                          lc_request_cb cb, void *user, uint64_t *req_id);

/* Delivers completed requests (callbacks), then starts queued ones that now fit.  Waits up to
 * timeout_ms for at least one completion while requests are in flight (0: do not wait).
 * *n_completed (may be NULL) receives the number delivered.  Errors: LC_ERR_ARG, LC_ERR_CUDA
 * (a request failed on the device; its callback received LC_ERR_CUDA). */
lc_status lc_serve_poll(lc_server *s, int timeout_ms, int *n_completed);

/* Cancels queued requests (callback status LC_ERR_STATE), waits for and delivers those on the
 * device, and frees the server (NULL is a no-op). */
lc_status lc_serve_close(lc_server *s);

/* Autotuner.  Chooses search parameters on a sample of queries q [n][d] (host float32) with
 * optional exact nearest-neighbour ids gt [n] (host int32; NULL: the top-1 of the plain search
 * at 4x efSearch stands in).  The plain FP32 search at tp->ef sets the 1-recall@1 target on
 * the sample.  Stage 1 tries every beam width 1, 2, 4 .. tp->max_beam with the FP32 and (if
 * tp->allow_fp16) the FP16 codebook, each at the smallest efSearch of the ladder
 * {2, 3, 4, 5, 6, 7, 8, 10, 12, 16} x ef/8 that reaches the target, and keeps the fastest.
 * Stage 2 times launch shapes for it (visited_log 0/10/11/12 x warps 0/4/8/12), which do not
 * change results, and keeps the fastest.  Times are medians of tp->reps searches of the
 * sample (repeated up to tp->batch queries) with device-resident queries (CUDA events; caches
 * stay warm between repetitions); recall counts each sample query once.
 * out->sp receives the parameters (k and shortlist as tp->k and the default), out->ms,
 * out->recall their time and recall on the sample, out->target and out->base_ms those of
 * the plain search at ef, out->tried the number of candidates timed.
 * Errors: LC_ERR_ARG, LC_ERR_STATE (untrained or empty index), LC_ERR_CUDA, LC_ERR_OOM. */
typedef struct {
    int k;           /* neighbours, 1..256 */
    int ef;          /* efSearch of the plain reference, 1..1024 */
    int allow_fp16;  /* 1: also try the FP16 level-1 codebook */
    int max_beam;    /* largest beam width tried, 1..8 (1: plain only) */
    int reps;        /* timed repetitions per candidate, >= 1 */
    int batch;       /* queries per timed search: the sample repeated up to this many (the batch
                        size the parameters are for: launch shapes that win on a small batch
                        can lose on a large one); 0 = the sample as it is */
} lc_tune_params;
typedef struct {
    lc_search_params sp;
    float ms, recall, target, base_ms;
    int tried;
} lc_tune_result;
lc_status lc_autotune(lc_index *ix, const float *q, int64_t n, const int32_t *gt, const lc_tune_params *tp,
                      lc_tune_result *out);

/* Captured search plans (the batched-serving form: one persistent walk kernel takes the
 * queries of a batch off a work queue; the whole search is recorded once into a CUDA graph).
 * lc_plan_create fixes the parameters *sp, the query type (LC_QUERY_F32 / LC_QUERY_U8) and
 * whether queries carry their own efSearch (per_query_ef: then every ef[i] must lie in
 * 1..sp->ef; values outside are clamped, as lc_search_ex with device arrays), allocates
 * device buffers for up to nq_max queries, and captures the search over them.  The index
 * must be non-empty; it is uploaded to the current device if needed.
 * lc_plan_buffers returns the plan's device buffers (any pointer may be NULL): q [nq_max][d]
 * (float32 or uint8), ef [nq_max] int32 (NULL without per_query_ef; initialised to sp->ef),
 * ids [nq_max][k], dists [nq_max][k], stats [nq_max][3], laid out as in lc_search.  The plan
 * owns them; they stay valid until lc_plan_free.
 * lc_plan_run queues one graph launch on `stream` for the first nq (0..nq_max) queries of
 * q; results are those lc_search(_ex) returns for the same queries and parameters.  Errors:
 * LC_ERR_STATE if the index was changed (lc_add, lc_import) or the current device differs
 * since the plan was made, LC_ERR_CUDA.  Runs of one plan must not overlap on the device
 * (they share the plan's buffers): queue them on one stream or wait in between.
 * lc_plan_free releases the plan; free plans before their index. */
typedef struct lc_plan lc_plan;
lc_status lc_plan_create(lc_index *ix, int64_t nq_max, const lc_search_params *sp, int qtype,
                         int per_query_ef, lc_plan **out);
lc_status lc_plan_buffers(const lc_plan *pl, void **q, int32_t **ef, int32_t **ids, float **dists,
                          int32_t **stats);
lc_status lc_plan_run(lc_plan *pl, int64_t nq, void *stream);
void lc_plan_free(lc_plan *pl);

/* Kernel timing: after lc_profile(ix, 1) every lc_search records CUDA events on its stream
 * around the walk kernel and the refinement kernel; lc_profile_read waits for the last
 * profiled search and returns the two durations in milliseconds (refine_ms = 0 without
 * refinement).  Uploads the index if needed.  Errors: LC_ERR_STATE (nothing profiled yet),
 * LC_ERR_CUDA. */
lc_status lc_profile(lc_index *ix, int enable);
lc_status lc_profile_read(lc_index *ix, float *walk_ms, float *refine_ms);

/* The last profiled search's phases, in milliseconds: the query rotation, the upper-level
 * descents and the queue sort of an ordered search (0 otherwise: the walk then descends
 * itself), the level-0 walk launch, and the refinement (0 without refinement).  walk_ms of
 * lc_profile_read is the sum of the first three.  Any pointer may be NULL.  Errors: as
 * lc_profile_read. */
lc_status lc_profile_phases(lc_index *ix, float *rotate_ms, float *descent_ms, float *level0_ms, float *refine_ms);

/* Frees the index and its device memory (NULL is a no-op). */
void lc_free(lc_index *ix);

/* Message of the last error on this thread ("" if none).  Valid until the next call. */
const char *lc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LC_H */
