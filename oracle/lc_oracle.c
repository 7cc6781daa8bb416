/*
 * Plain FP64 CPU oracle for the Link-and-Code search path and for the graph build that
 * produces the indexes it is checked on (Douze, Sablayrolles, Jegou, "Link and code: Fast
 * indexing with graphs and compact regression codes", CVPR 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the C-ABI library, its kernels or its
 * Python binding) may include, link or call this file.  It shares no code with them.  Only
 * the tests, the package entry point's smoke check and the benchmark's CPU-baseline leg use
 * it, through ctypes.
 *
 * Everything is single-threaded, in double precision, written for reading rather than
 * speed: sets are plain arrays scanned linearly, and each step follows the paper's order.
 *
 *   orc_search      Section 4.1 (two-stage search) over the HNSW structure of Section 2
 *                   (beam >= 2: the batched form, several expansions per step; tcap > 0:
 *                   stop after T level-0 distance computations, Section 3.1; C1w: the
 *                   codebook the walk's ADC terms use, NULL = C1; walk_full: the walk scores
 *                   the full two-level decode q(x) = c1 + c2 instead of the level-1 code,
 *                   with C2w standing for C2 as C1w for C1):
 *                   rotation, ADC tables, greedy descent of the upper levels, best-first
 *                   search of level 0, shortlist, refinement with the regression codebook
 *                   (Section 4.3, reconstruction beta^T G(x)), exact L2 and top-k.
 *   orc_build_graph HNSW insertion (Section 2 and Section 5.1: added by batches, distances
 *                   from the exact vector being inserted to the decoded indexed vectors).
 *
 * Ordering: every comparison is on the pair (distance, id), smaller id first on equal
 * distances.  orc_search also records, per query, the smallest relative gap between the two
 * distances of any comparison that decided its result: which node is expanded next (against
 * the runner-up and against the best node left outside the result set), when the walk ends,
 * where it moves on an upper level, the shortlist boundary and the order of the k returned.
 * A GPU run in FP32 may legitimately decide such a comparison the other way when that gap is
 * below its rounding error; every other comparison can change only the order inside the
 * result set, never the nodes expanded.  Two minima are reported: over every deciding
 * comparison, and over those that decide the walk and the shortlist only (not the order of
 * the k returned), so a query whose only near-tie is in its output order can still be held
 * to the same walk.  orc_trace lists the deciding comparisons one by one (for the tests that
 * pin this record against hand traces).
 *
 *   orc_dists       the walk distance and the refined distance of given (query, id) pairs,
 *                   computed directly from their definitions (no walk).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KBETA 8      /* neighbours in G(x), Section 4.2 */
#define ORC_NBETA 256    /* regression codebook size B, Section 4.3 */

/* ------------------------------------------------------------------------------------ */
/* Sub-space split: M contiguous blocks; the first (d mod M) have ceil(d/M) dimensions.    */
/* ------------------------------------------------------------------------------------ */
static void split_offsets(int d, int M, int *off, int *len)
{
    int base = d / M, extra = d % M, o = 0;
    for (int j = 0; j < M; j++) {
        len[j] = base + (j < extra ? 1 : 0);
        off[j] = o;
        o += len[j];
    }
}

/* Key order: (distance, id) lexicographic. */
static int key_less(double da, int32_t ia, double db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* Kinds of deciding comparison (orc_trace reports them with the two ids compared). */
enum {
    GAP_UPPER_SECOND = 1,   /* upper level: best neighbour against the runner-up */
    GAP_UPPER_MOVE = 2,     /* upper level: best neighbour against the current node */
    GAP_RUNNER = 3,         /* level 0: node expanded next against the runner-up in C */
    GAP_OUTSIDE = 4,        /* level 0: node expanded next against the best node outside W */
    GAP_BREAK = 5,          /* level 0: the furthest of W against the popped node that ends the walk */
    GAP_END = 6,            /* level 0: C ran empty; the worst of W against the best outside */
    GAP_BATCH_NEXT = 7,     /* batched: last member taken against the next unexpanded one */
    GAP_BATCH_OUTSIDE = 8,  /* batched: last member taken against the best node outside W */
    GAP_BATCH_END = 9,      /* batched: the worst of W against the best outside, at the end */
    GAP_SHORTLIST = 10,     /* the R-th of W against the (R+1)-th */
    GAP_OUT_WALK = 11,      /* output without refinement: consecutive returned, k-th vs (k+1)-th */
    GAP_OUT_REFINED = 12    /* output after refinement: the same on refined distances */
};

typedef struct {
    double gap;                 /* smallest relative gap seen so far, every kind */
    double gap_walk;            /* the same over the walk and shortlist kinds (1..10) */
    const uint8_t *codes1;      /* to recognise exact ties between identical code rows */
    int M1;
    const uint8_t *codes2;      /* non-NULL when the walk scores the full decode */
    int M2;
} gap_rec;

/* Trace of deciding comparisons (test use): (kind, first id, second id) triples. */
static _Thread_local int32_t *trace_buf = NULL;
static _Thread_local int trace_cap = 0;
static _Thread_local int trace_n = 0;

/* Starts (cap > 0) or stops (buf NULL) tracing on the calling thread; returns the number of
   triples written since the last start. */
int orc_trace(int32_t *buf, int cap)
{
    int n = trace_n;
    trace_buf = buf;
    trace_cap = buf ? cap : 0;
    trace_n = 0;
    return n;
}

static void note_gap(gap_rec *g, int kind, double a, int32_t ia, double b, int32_t ib)
{
    if (ia == ib) return;
    if (trace_buf && trace_n < trace_cap) {
        trace_buf[3 * trace_n] = kind;
        trace_buf[3 * trace_n + 1] = ia;
        trace_buf[3 * trace_n + 2] = ib;
        trace_n++;
    }
    double r;
    if (a == b) {
        /* Identical code rows give identical walk sums on any hardware; that tie is
           decided by id on both sides.  Any other exact tie is treated as unresolved. */
        int walk = kind != GAP_OUT_REFINED;
        if (walk && memcmp(g->codes1 + (int64_t)ia * g->M1, g->codes1 + (int64_t)ib * g->M1,
                           (size_t)g->M1) == 0 &&
            (!g->codes2 || memcmp(g->codes2 + (int64_t)ia * g->M2, g->codes2 + (int64_t)ib * g->M2,
                                  (size_t)g->M2) == 0))
            return;
        r = 0.0;
    } else {
        double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
        r = fabs(a - b) / m;
    }
    if (r < g->gap) g->gap = r;
    if (kind <= GAP_SHORTLIST && r < g->gap_walk) g->gap_walk = r;
}

static int cmp_note(gap_rec *g, int kind, double da, int32_t ia, double db, int32_t ib)
{
    note_gap(g, kind, da, ia, db, ib);
    return key_less(da, ia, db, ib);
}

/* ------------------------------------------------------------------------------------ */
/* Search                                                                               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t N;
    int d, M1, M2, deg, deg_up, max_level;
    int32_t ep;
    const float *R, *C1, *C2, *B;   /* B: [bM][bK][9] */
    int bM, bK;                      /* regression blocks, codewords per block */
    const uint8_t *codes1, *codes2, *beta;   /* beta: [N][bM] (unused when bK = 1) */
    const int32_t *adj0, *upper_off, *upper_adj;
} orc_index;

/* Walk distance by ADC (Section 4.1): the sum over level-1 sub-spaces of table entries,
   i.e. || y' - c1(x) ||^2 with the query unquantised and the database vector coded. */
static double adc(const orc_index *ix, const double *lut, int32_t e)
{
    const uint8_t *c = ix->codes1 + (int64_t)e * ix->M1;
    double s = 0.0;
    for (int j = 0; j < ix->M1; j++) s += lut[j * 256 + c[j]];
    return s;
}

/* What the walk scores a node by.  Level-1 walk (the default reading): the ADC sum above.
   Full walk: the squared distance to the node's full decode q(x) = c1(x) + c2(x), each
   coordinate t taking the level-1 centroid of its level-1 sub-space and the level-2 centroid
   of its level-2 sub-space (Section 4.1 describes the graph as searched with the codec's
   approximation; this is that approximation taken in full). */
typedef struct {
    const orc_index *ix;
    const double *lut;          /* ADC tables (level-1 walk) */
    int full;
    const double *yr;           /* rotated query (full walk) */
    const float *C1w, *C2w;     /* codebooks the full walk decodes with */
    const int *sub1, *sub2;     /* sub-space of each coordinate at level 1 and level 2 */
} walk_ctx;

static double wdist(const walk_ctx *w, int32_t e)
{
    if (!w->full) return adc(w->ix, w->lut, e);
    const orc_index *ix = w->ix;
    const uint8_t *a = ix->codes1 + (int64_t)e * ix->M1;
    const uint8_t *b = ix->codes2 + (int64_t)e * ix->M2;
    double s = 0.0;
    for (int t = 0; t < ix->d; t++) {
        double x = (double)w->C1w[(int64_t)a[w->sub1[t]] * ix->d + t] + (double)w->C2w[(int64_t)b[w->sub2[t]] * ix->d + t];
        double diff = w->yr[t] - x;
        s += diff * diff;
    }
    return s;
}

/* Decoded vector q(x) = c1(x) + c2(x - c1(x)) of the two-level codec (Section 3.3 / 4.1),
   in the rotated space. */
static void decode2(const orc_index *ix, const int *off1, const int *len1, const int *off2,
                    const int *len2, int32_t v, double *out)
{
    const uint8_t *a = ix->codes1 + (int64_t)v * ix->M1;
    const uint8_t *b = ix->codes2 + (int64_t)v * ix->M2;
    for (int j = 0; j < ix->M1; j++)
        for (int t = off1[j]; t < off1[j] + len1[j]; t++)
            out[t] = (double)ix->C1[(int64_t)a[j] * ix->d + t];
    for (int j = 0; j < ix->M2; j++)
        for (int t = off2[j]; t < off2[j] + len2[j]; t++)
            out[t] += (double)ix->C2[(int64_t)b[j] * ix->d + t];
}

/* Squared L2 from the rotated query yr to the refined reconstruction of node i (Section 4.2,
   4.3): y^ = sum_j beta_j q(v_j) over G = [q(i), q(g1..g8)], g the first 8 entries of i's
   level-0 row (a -1 entry is a zero column); with a product codebook each block of
   coordinates takes the weights of its own codeword.  xh, yh: scratch of d doubles (xh) and
   d doubles (yh). */
static double refined_dist(const orc_index *ix, const int *off1, const int *len1, const int *off2,
                           const int *len2, const int *offb, const int *lenb, const double *yr, int32_t i,
                           double *xh, double *yh)
{
    const int d = ix->d;
    for (int t = 0; t < d; t++) yh[t] = 0.0;
    for (int j = 0; j <= ORC_KBETA; j++) {
        int32_t v = j == 0 ? i : ix->adj0[(int64_t)i * ix->deg + (j - 1)];
        if (j > 0 && (j - 1 >= ix->deg || v < 0)) continue;     /* zero column */
        decode2(ix, off1, len1, off2, len2, v, xh);
        for (int m = 0; m < ix->bM; m++) {
            int b = ix->bK > 1 ? ix->beta[(int64_t)i * ix->bM + m] : 0;
            double w = (double)ix->B[((int64_t)m * ix->bK + b) * (ORC_KBETA + 1) + j];
            for (int t = offb[m]; t < offb[m] + lenb[m]; t++) yh[t] += w * xh[t];
        }
    }
    /* Exact squared L2 to the refined reconstruction */
    double s = 0.0;
    for (int t = 0; t < d; t++) {
        double diff = yr[t] - yh[t];
        s += diff * diff;
    }
    return s;
}

/* Level-0 search in the batched form: each step takes the `beam` best unexpanded members of
   W together, scores all their unvisited neighbours (a node shared by two rows is scored and
   counted once), and keeps the ef' best of W and the new nodes.  With beam = 1 this expands
   the same nodes in the same order as the best-first search of orc_search. */
static int walk_batched(const orc_index *ix, const walk_ctx *wc, int32_t seed, int efp, int beam,
                        int tcap, char *visited, int32_t *touched, int *ntouch, double *wd,
                        int32_t *wi, int32_t *n_dist, int32_t *n_expand, gap_rec *g)
{
    int cap = efp + beam * ix->deg + 1;
    double *ad = malloc(sizeof(double) * cap);
    int32_t *ai = malloc(sizeof(int32_t) * cap);
    char *af = malloc((size_t)cap);
    char *wf = calloc((size_t)efp + 1, 1);
    int32_t *U = malloc(sizeof(int32_t) * (beam > 0 ? beam : 1));
    int wn = 1;
    wd[0] = wdist(wc, seed);
    wi[0] = seed;
    visited[seed] = 1;
    touched[(*ntouch)++] = seed;
    *n_dist = 1;
    double od = INFINITY;              /* best scored node outside W */
    int32_t oi = -1;
    for (;;) {
        if (tcap > 0 && *n_dist >= tcap) break;          /* T distance computations done */
        int nu = 0;
        for (int p = 0; p < wn && nu < beam; p++)
            if (!wf[p]) U[nu++] = p;
        if (nu == 0) break;
        /* which members are taken is decided by the last one taken against the next
           unexpanded member and against the best node outside W */
        int last = U[nu - 1], next = -1;
        for (int p = last + 1; p < wn; p++)
            if (!wf[p]) { next = p; break; }
        if (nu == beam && next >= 0) note_gap(g, GAP_BATCH_NEXT, wd[last], wi[last], wd[next], wi[next]);
        /* with beam members taken, the best node outside W would be taken instead of the last
           one if it ranked before it; with fewer, every unexpanded member is taken and the
           outsider would be too if it ranked inside W at all (before its worst member) */
        if (oi >= 0 && nu == beam) note_gap(g, GAP_BATCH_OUTSIDE, wd[last], wi[last], od, oi);
        if (oi >= 0 && nu < beam) note_gap(g, GAP_BATCH_OUTSIDE, wd[wn - 1], wi[wn - 1], od, oi);
        int an = 0;
        for (int p = 0; p < wn; p++) { ad[an] = wd[p]; ai[an] = wi[p]; af[an] = wf[p]; an++; }
        for (int u = 0; u < nu; u++) af[U[u]] = 1;
        *n_expand += nu;
        for (int u = 0; u < nu; u++) {
            const int32_t *row = ix->adj0 + (int64_t)wi[U[u]] * ix->deg;
            for (int s2 = 0; s2 < ix->deg; s2++) {
                int32_t e = row[s2];
                if (e < 0 || visited[e]) continue;
                visited[e] = 1;
                touched[(*ntouch)++] = e;
                (*n_dist)++;
                ad[an] = wdist(wc, e); ai[an] = e; af[an] = 0; an++;
            }
        }
        /* order W and the new nodes by key (insertion sort) and keep the ef' best */
        for (int x = 1; x < an; x++) {
            double dx = ad[x]; int32_t ix2 = ai[x]; char fx = af[x];
            int y = x;
            while (y > 0 && key_less(dx, ix2, ad[y - 1], ai[y - 1])) {
                ad[y] = ad[y - 1]; ai[y] = ai[y - 1]; af[y] = af[y - 1];
                y--;
            }
            ad[y] = dx; ai[y] = ix2; af[y] = fx;
        }
        wn = an < efp ? an : efp;
        if (an > efp && key_less(ad[efp], ai[efp], od, oi < 0 ? INT32_MAX : oi)) {
            od = ad[efp]; oi = ai[efp];
        }
        for (int p = 0; p < wn; p++) { wd[p] = ad[p]; wi[p] = ai[p]; wf[p] = af[p]; }
    }
    /* the end (every member expanded, or the cap T reached): the best node outside W
       against the worst inside decides whether the walk had a member left to take, and
       which nodes W holds */
    if (oi >= 0) note_gap(g, GAP_BATCH_END, wd[wn - 1], wi[wn - 1], od, oi);
    free(ad); free(ai); free(af); free(wf); free(U);
    return wn;
}

int orc_search(int64_t N, int d, int M1, int M2, const float *R, const float *C1,
               const float *C2, const uint8_t *codes1, const uint8_t *codes2,
               const uint8_t *beta, const float *B, int bM, int bK, int deg, const int32_t *adj0, int deg_up,
               const int32_t *upper_off, const int32_t *upper_adj, int32_t ep, int max_level,
               int64_t nq, const float *Q, int k, int ef, int shortlist, int beam, int tcap,
               const float *C1w, int walk_full, const float *C2w, int32_t *ids, double *dists,
               int32_t *stats, double *min_gap, double *min_gap_walk, double *next_dist,
               int32_t *w_ids, double *w_dists, int32_t *w_size)
{
    orc_index ix = {N, d, M1, M2, deg, deg_up, max_level, ep, R, C1, C2, B, bM, bK,
                    codes1, codes2, beta, adj0, upper_off, upper_adj};
    int efp = ef > k ? ef : k;                               /* ef' = max(efSearch, k) */
    /* the walk's codebook: C1 itself, or a variant of it (e.g. rounded to FP16); the
       refinement always decodes with C1 */
    if (!C1w) C1w = C1;
    if (!C2w) C2w = C2;
    int off1[256], len1[256], off2[256], len2[256], offb[256], lenb[256];
    if (M1 > 256 || M2 > 256 || bM < 1 || bM > 256 || bM > d || bK < 1 || bK > 256 || k < 1) return -1;
    split_offsets(d, M1, off1, len1);
    split_offsets(d, M2, off2, len2);
    split_offsets(d, bM, offb, lenb);       /* regression blocks (Section 4.3, product codebook) */
    int *sub1 = malloc(sizeof(int) * d), *sub2 = malloc(sizeof(int) * d);
    for (int j = 0; j < M1; j++) for (int t = off1[j]; t < off1[j] + len1[j]; t++) sub1[t] = j;
    for (int j = 0; j < M2; j++) for (int t = off2[j]; t < off2[j] + len2[j]; t++) sub2[t] = j;

    double *yr = malloc(sizeof(double) * d);
    double *lut = malloc(sizeof(double) * 256 * M1);
    char *visited = N > 0 ? calloc((size_t)N, 1) : NULL;
    int32_t *touched = malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    int64_t cap = (int64_t)efp * 4 + (int64_t)deg * 4 + 16;
    double *cd = malloc(sizeof(double) * cap);               /* candidate set C */
    int32_t *ci = malloc(sizeof(int32_t) * cap);
    double *wd = malloc(sizeof(double) * (efp + 1));         /* result set W */
    int32_t *wi = malloc(sizeof(int32_t) * (efp + 1));
    double *xh = malloc(sizeof(double) * d * (ORC_KBETA + 1));
    double *yh = malloc(sizeof(double) * d);
    double *rd = malloc(sizeof(double) * (efp + 1));
    int32_t *ri = malloc(sizeof(int32_t) * (efp + 1));

    for (int64_t q = 0; q < nq; q++) {
        const float *y = Q + q * d;
        gap_rec g = {INFINITY, INFINITY, codes1, M1, walk_full ? codes2 : NULL, M2};
        walk_ctx wc = {&ix, lut, walk_full, yr, C1w, C2w, sub1, sub2};
        int32_t n_dist = 0, n_expand = 0, n_up = 0;
        int wn = 0, ntouch = 0;

        /* Rotation y' = R y (orthogonal, so L2 distances are unchanged). */
        for (int t = 0; t < d; t++) {
            double s = 0.0;
            for (int u = 0; u < d; u++) s += (double)R[(int64_t)t * d + u] * (double)y[u];
            yr[t] = s;
        }
        /* ADC tables LUT[j][c] = || y'^j - C1_j[c] ||^2, in difference form. */
        for (int j = 0; j < M1 && !walk_full; j++)
            for (int c = 0; c < 256; c++) {
                double s = 0.0;
                for (int t = off1[j]; t < off1[j] + len1[j]; t++) {
                    double diff = yr[t] - (double)C1w[(int64_t)c * d + t];
                    s += diff * diff;
                }
                lut[j * 256 + c] = s;
            }

        if (N > 0) {
            /* Greedy descent through levels max_level..1 (Section 2). */
            int32_t cur = ep;
            double dcur = wdist(&wc, cur);
            if (max_level >= 1) n_up++;
            for (int l = max_level; l >= 1; l--) {
                for (;;) {
                    const int32_t *row = upper_adj + ((int64_t)upper_off[cur] + l - 1) * deg_up;
                    int32_t best = -1, second = -1;
                    double dbest = 0.0, dsecond = 0.0;
                    for (int s = 0; s < deg_up; s++) {
                        int32_t e = row[s];
                        if (e < 0) continue;
                        double de = wdist(&wc, e);
                        n_up++;
                        if (best < 0 || key_less(de, e, dbest, best)) {
                            second = best; dsecond = dbest;
                            best = e; dbest = de;
                        } else if (second < 0 || key_less(de, e, dsecond, second)) {
                            second = e; dsecond = de;
                        }
                    }
                    /* deciding comparisons: the best neighbour against the runner-up,
                       and against the current node */
                    if (second >= 0) note_gap(&g, GAP_UPPER_SECOND, dbest, best, dsecond, second);
                    if (best >= 0 && cmp_note(&g, GAP_UPPER_MOVE, dbest, best, dcur, cur)) {
                        cur = best;
                        dcur = dbest;
                    } else {
                        break;
                    }
                }
            }

            if (beam >= 2) {
                wn = walk_batched(&ix, &wc, cur, efp, beam, tcap, visited, touched, &ntouch, wd, wi,
                                  &n_dist, &n_expand, &g);
            } else {
                /* Best-first search of level 0 from the seed, result set of size ef'. */
                int64_t cn = 0;
                double d0 = wdist(&wc, cur);
                n_dist = 1;
                visited[cur] = 1;
                touched[ntouch++] = cur;
                cd[cn] = d0; ci[cn] = cur; cn++;
                wd[0] = d0; wi[0] = cur; wn = 1;
                /* best node scored so far that is not in W (rejected or evicted); W is always
                   the ef' best scored nodes, so this is the (ef'+1)-th best */
                double od0 = INFINITY;
                int32_t oid = -1;
                while (cn > 0) {
                    /* the search-time cap T of Section 3.1: stop once T distance
                       computations have been made (checked before each expansion) */
                    if (tcap > 0 && n_dist >= tcap) break;
                    /* c = nearest element of C; its order against the runner-up decides
                       which element is expanded first */
                    int64_t bc = 0, b2 = -1;
                    for (int64_t s = 1; s < cn; s++) {
                        if (key_less(cd[s], ci[s], cd[bc], ci[bc])) { b2 = bc; bc = s; }
                        else if (b2 < 0 || key_less(cd[s], ci[s], cd[b2], ci[b2])) b2 = s;
                    }
                    if (b2 >= 0) note_gap(&g, GAP_RUNNER, cd[bc], ci[bc], cd[b2], ci[b2]);
                    double dc = cd[bc];
                    int32_t c = ci[bc];
                    cd[bc] = cd[cn - 1]; ci[bc] = ci[cn - 1]; cn--;
                    /* f = furthest element of W */
                    int bf = 0;
                    for (int s = 1; s < wn; s++)
                        if (key_less(wd[bf], wi[bf], wd[s], wi[s])) bf = s;
                    if (key_less(wd[bf], wi[bf], dc, c)) {                 /* c further than f */
                        note_gap(&g, GAP_BREAK, wd[bf], wi[bf], dc, c);
                        break;
                    }
                    /* c is expanded next: decided against the runner-up in C (above) and
                       against the best node outside W */
                    if (oid >= 0) note_gap(&g, GAP_OUTSIDE, dc, c, od0, oid);
                    n_expand++;
                    const int32_t *row = adj0 + (int64_t)c * deg;
                    for (int s = 0; s < deg; s++) {
                        int32_t e = row[s];
                        if (e < 0 || visited[e]) continue;
                        visited[e] = 1;
                        touched[ntouch++] = e;
                        double de = wdist(&wc, e);
                        n_dist++;
                        bf = 0;
                        for (int u = 1; u < wn; u++)
                            if (key_less(wd[bf], wi[bf], wd[u], wi[u])) bf = u;
                        int take = wn < efp || key_less(de, e, wd[bf], wi[bf]);
                        if (!take && key_less(de, e, od0, oid < 0 ? INT32_MAX : oid)) {
                            od0 = de; oid = e;
                        }
                        if (take) {
                            if (cn == cap) {
                                cap *= 2;
                                cd = realloc(cd, sizeof(double) * cap);
                                ci = realloc(ci, sizeof(int32_t) * cap);
                            }
                            cd[cn] = de; ci[cn] = e; cn++;
                            wd[wn] = de; wi[wn] = e; wn++;
                            if (wn > efp) {                      /* evict the furthest */
                                int s1 = 0;
                                for (int u = 1; u < wn; u++)
                                    if (key_less(wd[s1], wi[s1], wd[u], wi[u])) s1 = u;
                                if (key_less(wd[s1], wi[s1], od0, oid < 0 ? INT32_MAX : oid)) {
                                    od0 = wd[s1]; oid = wi[s1];
                                }
                                wd[s1] = wd[wn - 1]; wi[s1] = wi[wn - 1]; wn--;
                            }
                        }
                    }
                }
                /* the end, however it came (C empty, a popped node beyond the worst of W, or
                   the cap T): had the best node outside W ranked inside it, the walk would
                   have had it to expand (the result-list view: W holds an unexpanded member),
                   and W's members would differ */
                if (oid >= 0) {
                    int bf = 0;
                    for (int s = 1; s < wn; s++)
                        if (key_less(wd[bf], wi[bf], wd[s], wi[s])) bf = s;
                    note_gap(&g, GAP_END, wd[bf], wi[bf], od0, oid);
                }
            }
            for (int s = 0; s < ntouch; s++) visited[touched[s]] = 0;

            /* sort W by (distance, id) */
            for (int a = 0; a < wn; a++) {
                int m = a;
                for (int b2 = a + 1; b2 < wn; b2++)
                    if (key_less(wd[b2], wi[b2], wd[m], wi[m])) m = b2;
                double td = wd[a]; wd[a] = wd[m]; wd[m] = td;
                int32_t ti = wi[a]; wi[a] = wi[m]; wi[m] = ti;
            }
        }

        if (w_size) w_size[q] = wn;
        if (w_ids)
            for (int s = 0; s < efp; s++) {
                w_ids[q * efp + s] = s < wn ? wi[s] : -1;
                w_dists[q * efp + s] = s < wn ? wd[s] : INFINITY;
            }

        int32_t *oi = ids + q * k;
        double *od = dists + q * k;
        for (int s = 0; s < k; s++) { oi[s] = -1; od[s] = INFINITY; }
        double nd = INFINITY;           /* the distance that follows the k returned */

        if (shortlist < 0) {
            /* no refinement: top-k of W by walk distance; the order of the k returned
               and the k-th against the (k+1)-th decide the output */
            for (int s = 0; s < k && s < wn; s++) {
                oi[s] = wi[s]; od[s] = wd[s];
                if (s + 1 < wn) note_gap(&g, GAP_OUT_WALK, wd[s], wi[s], wd[s + 1], wi[s + 1]);
            }
            if (k < wn) nd = wd[k];
        } else {
            /* Shortlist R = the R best of W (at most 10 refined by default, Sec. 5.1);
               the R-th against the (R+1)-th decides its membership */
            int Rn = shortlist > 0 ? shortlist : 10;
            if (Rn < k) Rn = k;
            if (Rn > wn) Rn = wn;
            if (Rn > 0 && Rn < wn) note_gap(&g, GAP_SHORTLIST, wd[Rn - 1], wi[Rn - 1], wd[Rn], wi[Rn]);
            /* Refined reconstruction y^ = sum_j beta_j q(v_j), G = [q(x), q(g1..g8)]; with a
               product codebook each block of coordinates takes the weights of its own
               codeword (one codeword per block: the shared 0-byte weights) */
            for (int r = 0; r < Rn; r++) {
                rd[r] = refined_dist(&ix, off1, len1, off2, len2, offb, lenb, yr, wi[r], xh, yh);
                ri[r] = wi[r];
            }
            for (int a = 0; a < Rn; a++) {
                int m = a;
                for (int b2 = a + 1; b2 < Rn; b2++)
                    if (key_less(rd[b2], ri[b2], rd[m], ri[m])) m = b2;
                double td = rd[a]; rd[a] = rd[m]; rd[m] = td;
                int32_t ti = ri[a]; ri[a] = ri[m]; ri[m] = ti;
            }
            /* the order of the k returned, and the k-th against the (k+1)-th */
            for (int s = 0; s < k && s < Rn; s++) {
                oi[s] = ri[s]; od[s] = rd[s];
                if (s + 1 < Rn) note_gap(&g, GAP_OUT_REFINED, rd[s], ri[s], rd[s + 1], ri[s + 1]);
            }
            if (k < Rn) nd = rd[k];
        }
        if (stats) {
            stats[q * 3 + 0] = n_dist;
            stats[q * 3 + 1] = n_expand;
            stats[q * 3 + 2] = n_up;
        }
        if (min_gap) min_gap[q] = g.gap;
        if (min_gap_walk) min_gap_walk[q] = g.gap_walk;
        if (next_dist) next_dist[q] = nd;
    }
    free(yr); free(lut); free(sub1); free(sub2); free(visited); free(touched); free(cd); free(ci);
    free(wd); free(wi); free(xh); free(yh); free(rd); free(ri);
    return 0;
}

/* Walk distance and refined distance of m given ids per query, from their definitions
   (rotation, ADC table or full decode, refined reconstruction), without any walk: for
   checking a result list id by id.  ids [nq][m] (-1 gives +inf); walk_d, ref_d [nq][m]. */
int orc_dists(int64_t N, int d, int M1, int M2, const float *R, const float *C1,
              const float *C2, const uint8_t *codes1, const uint8_t *codes2,
              const uint8_t *beta, const float *B, int bM, int bK, int deg, const int32_t *adj0,
              int64_t nq, const float *Q, int m, const int32_t *ids, const float *C1w, int walk_full,
              const float *C2w, double *walk_d, double *ref_d)
{
    orc_index ix = {N, d, M1, M2, deg, 0, 0, -1, R, C1, C2, B, bM, bK,
                    codes1, codes2, beta, adj0, NULL, NULL};
    if (!C1w) C1w = C1;
    if (!C2w) C2w = C2;
    int off1[256], len1[256], off2[256], len2[256], offb[256], lenb[256];
    if (M1 > 256 || M2 > 256 || bM < 1 || bM > 256 || bM > d || bK < 1 || bK > 256) return -1;
    split_offsets(d, M1, off1, len1);
    split_offsets(d, M2, off2, len2);
    split_offsets(d, bM, offb, lenb);
    int *sub1 = malloc(sizeof(int) * d), *sub2 = malloc(sizeof(int) * d);
    for (int j = 0; j < M1; j++) for (int t = off1[j]; t < off1[j] + len1[j]; t++) sub1[t] = j;
    for (int j = 0; j < M2; j++) for (int t = off2[j]; t < off2[j] + len2[j]; t++) sub2[t] = j;
    double *yr = malloc(sizeof(double) * d);
    double *lut = malloc(sizeof(double) * 256 * M1);
    double *xh = malloc(sizeof(double) * d);
    double *yh = malloc(sizeof(double) * d);
    for (int64_t q = 0; q < nq; q++) {
        const float *y = Q + q * d;
        walk_ctx wc = {&ix, lut, walk_full, yr, C1w, C2w, sub1, sub2};
        for (int t = 0; t < d; t++) {
            double s = 0.0;
            for (int u = 0; u < d; u++) s += (double)R[(int64_t)t * d + u] * (double)y[u];
            yr[t] = s;
        }
        for (int j = 0; j < M1 && !walk_full; j++)
            for (int c = 0; c < 256; c++) {
                double s = 0.0;
                for (int t = off1[j]; t < off1[j] + len1[j]; t++) {
                    double diff = yr[t] - (double)C1w[(int64_t)c * d + t];
                    s += diff * diff;
                }
                lut[j * 256 + c] = s;
            }
        for (int r = 0; r < m; r++) {
            int32_t i = ids[q * m + r];
            if (i < 0 || i >= N) {
                walk_d[q * m + r] = INFINITY;
                ref_d[q * m + r] = INFINITY;
                continue;
            }
            walk_d[q * m + r] = wdist(&wc, i);
            ref_d[q * m + r] = refined_dist(&ix, off1, len1, off2, len2, offb, lenb, yr, i, xh, yh);
        }
    }
    free(sub1); free(sub2); free(yr); free(lut); free(xh); free(yh);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Graph build                                                                          */
/* ------------------------------------------------------------------------------------ */
/*
 * Inputs: xr = exact vectors (rotated), xh = their two-level decodings, both [N][d];
 * levels[i] = the level of node i.  Points are inserted in id order, in batches: a batch
 * of size b = max(1, min(batch_max, n / batch_div)) starts when n nodes are in the graph;
 * every point of the batch searches the graph as it stood at the start of the batch, then
 * the links are applied in id order.  With batch_max = 1 every batch holds one point and
 * this is plain sequential insertion.
 *
 * Distances: from the point being inserted, exact-to-decoded (Section 4.1: the vector to
 * insert is not quantised, the indexed ones are); between two indexed points, decoded to
 * decoded.  Each row is kept sorted by (decoded-to-decoded distance to its owner, id).
 * Neighbour selection is the shrinking heuristic of HNSW (Section 2): a candidate is kept
 * unless an already kept neighbour is closer to it than the base point is.
 */
typedef struct {
    int32_t *id;   /* [rows][M] */
    double *dist;  /* [rows][M] */
    int32_t *cnt;  /* [rows] */
    int M;
} rowset;

static double l2(const double *a, const double *b, int d)
{
    double s = 0.0;
    for (int t = 0; t < d; t++) {
        double x = a[t] - b[t];
        s += x * x;
    }
    return s;
}

typedef struct {
    int64_t N;
    int d;
    const double *xr, *xh;
    rowset lev0, up;
    const int32_t *upper_off;
} orc_graph;

static int32_t *row_ids(orc_graph *g, int l, int32_t v, int *cnt, int *M)
{
    if (l == 0) {
        *cnt = g->lev0.cnt[v]; *M = g->lev0.M;
        return g->lev0.id + (int64_t)v * g->lev0.M;
    }
    int64_t r = (int64_t)g->upper_off[v] + l - 1;
    *cnt = g->up.cnt[r]; *M = g->up.M;
    return g->up.id + r * g->up.M;
}

/* Best-first search of one level from `entry`, keeping the ef closest: the same layer
   search as the query path, with exact-to-decoded distances.  Output sorted by key. */
static int search_layer(orc_graph *g, const double *x, int32_t entry, int ef, int l,
                        char *visited, int32_t *touched, double *cd, int32_t *ci,
                        double *wd, int32_t *wi)
{
    int64_t cn = 0, nt = 0;
    int wn = 0;
    double d0 = l2(x, g->xh + (int64_t)entry * g->d, g->d);
    visited[entry] = 1; touched[nt++] = entry;
    cd[cn] = d0; ci[cn] = entry; cn++;
    wd[0] = d0; wi[0] = entry; wn = 1;
    while (cn > 0) {
        int64_t bc = 0;
        for (int64_t s = 1; s < cn; s++)
            if (key_less(cd[s], ci[s], cd[bc], ci[bc])) bc = s;
        double dc = cd[bc];
        int32_t c = ci[bc];
        cd[bc] = cd[cn - 1]; ci[bc] = ci[cn - 1]; cn--;
        int bf = 0;
        for (int s = 1; s < wn; s++)
            if (key_less(wd[bf], wi[bf], wd[s], wi[s])) bf = s;
        if (key_less(wd[bf], wi[bf], dc, c)) break;
        int cnt, M;
        int32_t *row = row_ids(g, l, c, &cnt, &M);
        for (int s = 0; s < cnt; s++) {
            int32_t e = row[s];
            if (visited[e]) continue;
            visited[e] = 1; touched[nt++] = e;
            double de = l2(x, g->xh + (int64_t)e * g->d, g->d);
            bf = 0;
            for (int u = 1; u < wn; u++)
                if (key_less(wd[bf], wi[bf], wd[u], wi[u])) bf = u;
            if (wn < ef || key_less(de, e, wd[bf], wi[bf])) {
                cd[cn] = de; ci[cn] = e; cn++;
                wd[wn] = de; wi[wn] = e; wn++;
                if (wn > ef) {
                    bf = 0;
                    for (int u = 1; u < wn; u++)
                        if (key_less(wd[bf], wi[bf], wd[u], wi[u])) bf = u;
                    wd[bf] = wd[wn - 1]; wi[bf] = wi[wn - 1]; wn--;
                }
            }
        }
    }
    for (int64_t s = 0; s < nt; s++) visited[touched[s]] = 0;
    for (int a = 0; a < wn; a++) {
        int m = a;
        for (int b = a + 1; b < wn; b++)
            if (key_less(wd[b], wi[b], wd[m], wi[m])) m = b;
        double td = wd[a]; wd[a] = wd[m]; wd[m] = td;
        int32_t ti = wi[a]; wi[a] = wi[m]; wi[m] = ti;
    }
    return wn;
}

/* Shrinking heuristic: candidates (cd, ci) sorted by key w.r.t. the base point; keep e
   unless some kept k has ||x^_e - x^_k||^2 < dist(base, e).  At most M kept. */
static int heuristic(orc_graph *g, const double *cd, const int32_t *ci, int n, int M,
                     int32_t *out)
{
    int kept = 0;
    for (int s = 0; s < n && kept < M; s++) {
        const double *xe = g->xh + (int64_t)ci[s] * g->d;
        int good = 1;
        for (int u = 0; u < kept; u++)
            if (l2(xe, g->xh + (int64_t)out[u] * g->d, g->d) < cd[s]) { good = 0; break; }
        if (good) out[kept++] = ci[s];
    }
    return kept;
}

/* Insert (id, dist) into a row kept sorted by (dist, id); on overflow, re-select the
   row's members plus the newcomer with the heuristic. */
static void add_link(orc_graph *g, int l, int32_t owner, int32_t x)
{
    rowset *rs = l == 0 ? &g->lev0 : &g->up;
    int64_t r = l == 0 ? owner : (int64_t)g->upper_off[owner] + l - 1;
    int32_t *id = rs->id + r * rs->M;
    double *ds = rs->dist + r * rs->M;
    int n = rs->cnt[r];
    double dx = l2(g->xh + (int64_t)owner * g->d, g->xh + (int64_t)x * g->d, g->d);
    for (int s = 0; s < n; s++) if (id[s] == x) return;
    /* merged candidate list, sorted */
    double cd[257];
    int32_t ci[257];
    int m = 0, ins = 0;
    for (int s = 0; s < n; s++) {
        if (!ins && key_less(dx, x, ds[s], id[s])) { cd[m] = dx; ci[m] = x; m++; ins = 1; }
        cd[m] = ds[s]; ci[m] = id[s]; m++;
    }
    if (!ins) { cd[m] = dx; ci[m] = x; m++; }
    if (m <= rs->M) {
        for (int s = 0; s < m; s++) { id[s] = ci[s]; ds[s] = cd[s]; }
        rs->cnt[r] = m;
        return;
    }
    int32_t keep[256];
    int kn = heuristic(g, cd, ci, m, rs->M, keep);
    /* keep[] is in candidate order, i.e. still sorted by key */
    int s2 = 0;
    for (int s = 0; s < m && s2 < kn; s++)
        if (ci[s] == keep[s2]) { id[s2] = ci[s]; ds[s2] = cd[s]; s2++; }
    rs->cnt[r] = kn;
}

int orc_build_graph(int64_t N, int d, const double *xr, const double *xh,
                    const int32_t *levels, int deg, int deg_up, int efc, int batch_max,
                    int batch_div, int32_t *adj0, const int32_t *upper_off,
                    int64_t n_upper_rows, int32_t *upper_adj, int32_t *ep_out,
                    int32_t *maxlev_out)
{
    if (deg > 256 || deg_up > 256 || efc < 1) return -1;
    orc_graph g;
    g.N = N; g.d = d; g.xr = xr; g.xh = xh; g.upper_off = upper_off;
    g.lev0.M = deg;
    g.lev0.id = malloc(sizeof(int32_t) * (N > 0 ? N : 1) * deg);
    g.lev0.dist = malloc(sizeof(double) * (N > 0 ? N : 1) * deg);
    g.lev0.cnt = calloc((size_t)(N > 0 ? N : 1), sizeof(int32_t));
    g.up.M = deg_up;
    g.up.id = malloc(sizeof(int32_t) * (n_upper_rows > 0 ? n_upper_rows : 1) * deg_up);
    g.up.dist = malloc(sizeof(double) * (n_upper_rows > 0 ? n_upper_rows : 1) * deg_up);
    g.up.cnt = calloc((size_t)(n_upper_rows > 0 ? n_upper_rows : 1), sizeof(int32_t));

    char *visited = calloc((size_t)(N > 0 ? N : 1), 1);
    int32_t *touched = malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    int64_t cap = N + 1;   /* C never holds more than the visited nodes */
    double *cd = malloc(sizeof(double) * cap);
    int32_t *ci = malloc(sizeof(int32_t) * cap);
    double *wd = malloc(sizeof(double) * (efc + 1));
    int32_t *wi = malloc(sizeof(int32_t) * (efc + 1));

    int32_t ep = -1;
    int maxlev = -1;
    int64_t n = 0;
    int maxbatch = batch_max > 0 ? batch_max : 1;
    /* per batch member: selected neighbours per level (levels are below 32) */
    int Mx = deg > deg_up ? deg : deg_up;
    int32_t *sel = malloc(sizeof(int32_t) * (int64_t)maxbatch * 32 * Mx);
    int *seln = malloc(sizeof(int) * (int64_t)maxbatch * 32);

    while (n < N) {
        int64_t b = batch_div > 0 ? n / batch_div : 1;
        if (b > batch_max) b = batch_max;
        if (b < 1) b = 1;
        if (n + b > N) b = N - n;
        if (n == 0) b = 1;
        int ml0 = maxlev;
        int32_t ep0 = ep;
        for (int64_t u = 0; u < b; u++) {
            int64_t x = n + u;
            const double *xv = xr + x * d;
            int Lx = levels[x];
            for (int l = 0; l < 32; l++) seln[u * 32 + l] = 0;
            if (ep0 < 0) continue;
            int32_t cur = ep0;
            double dcur = l2(xv, xh + (int64_t)cur * d, d);
            for (int l = ml0; l > Lx; l--) {
                for (;;) {
                    int cnt, M;
                    int32_t *row = row_ids(&g, l, cur, &cnt, &M);
                    int32_t best = -1;
                    double dbest = 0.0;
                    for (int s = 0; s < cnt; s++) {
                        double de = l2(xv, xh + (int64_t)row[s] * d, d);
                        if (best < 0 || key_less(de, row[s], dbest, best)) {
                            best = row[s]; dbest = de;
                        }
                    }
                    if (best >= 0 && key_less(dbest, best, dcur, cur)) { cur = best; dcur = dbest; }
                    else break;
                }
            }
            for (int l = (Lx < ml0 ? Lx : ml0); l >= 0; l--) {
                int wn = search_layer(&g, xv, cur, efc, l, visited, touched, cd, ci, wd, wi);
                int M = l == 0 ? deg : deg_up;
                seln[u * 32 + l] = heuristic(&g, wd, wi, wn, M, sel + ((int64_t)u * 32 + l) * Mx);
                cur = wi[0];
            }
        }
        /* links, in id order */
        for (int64_t u = 0; u < b; u++) {
            int64_t x = n + u;
            int Lx = levels[x];
            for (int l = 0; l <= Lx && l <= ml0; l++) {
                int32_t *sx = sel + ((int64_t)u * 32 + l) * Mx;
                int cnt = seln[u * 32 + l];
                /* the new node's own row, sorted by decoded-to-decoded distance */
                rowset *rs = l == 0 ? &g.lev0 : &g.up;
                int64_t r = l == 0 ? x : (int64_t)upper_off[x] + l - 1;
                int m = 0;
                for (int s = 0; s < cnt; s++) {
                    double dv = l2(xh + x * d, xh + (int64_t)sx[s] * d, d);
                    int p = m;
                    while (p > 0 && key_less(dv, sx[s], rs->dist[r * rs->M + p - 1],
                                             rs->id[r * rs->M + p - 1])) {
                        rs->dist[r * rs->M + p] = rs->dist[r * rs->M + p - 1];
                        rs->id[r * rs->M + p] = rs->id[r * rs->M + p - 1];
                        p--;
                    }
                    rs->dist[r * rs->M + p] = dv;
                    rs->id[r * rs->M + p] = sx[s];
                    m++;
                }
                rs->cnt[r] = m;
            }
        }
        for (int64_t u = 0; u < b; u++) {
            int64_t x = n + u;
            int Lx = levels[x];
            for (int l = 0; l <= Lx && l <= ml0; l++) {
                int32_t *sx = sel + ((int64_t)u * 32 + l) * Mx;
                for (int s = 0; s < seln[u * 32 + l]; s++) add_link(&g, l, sx[s], (int32_t)x);
            }
        }
        for (int64_t u = 0; u < b; u++) {
            int64_t x = n + u;
            if (levels[x] > maxlev) { maxlev = levels[x]; ep = (int32_t)x; }
        }
        n += b;
    }

    for (int64_t i = 0; i < N; i++)
        for (int s = 0; s < deg; s++)
            adj0[i * deg + s] = s < g.lev0.cnt[i] ? g.lev0.id[i * deg + s] : -1;
    for (int64_t r = 0; r < n_upper_rows; r++)
        for (int s = 0; s < deg_up; s++)
            upper_adj[r * deg_up + s] = s < g.up.cnt[r] ? g.up.id[r * deg_up + s] : -1;
    *ep_out = ep;
    *maxlev_out = maxlev < 0 ? 0 : maxlev;

    free(g.lev0.id); free(g.lev0.dist); free(g.lev0.cnt);
    free(g.up.id); free(g.up.dist); free(g.up.cnt);
    free(visited); free(touched); free(cd); free(ci); free(wd); free(wi);
    free(sel); free(seln);
    return 0;
}
