// Host build of a Link-and-Code index: codec training, encoding, HNSW insertion and the
// regression codebook (Douze, Sablayrolles, Jegou, CVPR 2018).
//
//  * Codec (Section 3.3, 4.1, 5.1): level 1 = (O)PQ M1 x 8 on x' = R x, level 2 = PQ M2 x 8
//    on the residual x' - c1(x'); q(x) = c1 + c2.  OPQ alternates a PQ k-means step in the
//    rotated space with the orthogonal Procrustes update R = U V^T (computed as the polar
//    factor M (M^T M)^{-1/2} with a Jacobi eigen-solver).
//  * Graph (Section 2, 4.1, 5.1): HNSW levels with ratio 30 between level sizes, degree 32,
//    points inserted by batches; every point of a batch searches the graph as it stood at
//    the start of the batch (in parallel), then links are applied in id order.  Distances
//    from the inserted vector are exact-to-decoded (the inserted vector is not quantised);
//    distances between indexed vectors are decoded-to-decoded.  Neighbours are chosen with
//    HNSW's shrinking heuristic; rows are kept sorted by distance to their owner, so the
//    first 8 entries are the neighbours g_1..g_8 of G(x) "ordered by increasing distance".
//  * Regression codebook (Section 4.3): k-means on per-vector least-squares weights to
//    initialise, then EM (assignment by argmin of ||x - beta^T G(x)||^2, per-cluster least
//    squares); codeword 0 is e0 = (1, 0, ..., 0) and is never updated, so no vector is
//    refined worse than q(x).  Trained on a seeded subset of at most 250k vectors.
//
// This is the build side of the library; the search path runs on the GPU (lc_search.cu), and
// with build_gpu = 1 the level-0 insertions of each batch do too (lc_build_gpu.cu).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>
#include <utility>

#include <cuda_runtime.h>

#include "lc_internal.h"

namespace lc {

int n_threads(const lc_params &p)
{
    int t = p.n_threads > 0 ? p.n_threads : (int)std::thread::hardware_concurrency();
    return t < 1 ? 1 : t;
}

// Runs f(begin, end, thread) over [0, n) in chunks handed out dynamically.  Each index is
// processed by a pure function of shared read-only state, so the result does not depend
// on the scheduling.
template <class F>
static void parallel_for(int64_t n, int nt, int64_t chunk, F &&f)
{
    if (n <= 0) return;
    if (chunk < 1) chunk = 1;
    int64_t nchunks = (n + chunk - 1) / chunk;
    if (nt > nchunks) nt = (int)nchunks;
    if (nt <= 1) {
        f((int64_t)0, n, 0);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            for (;;) {
                int64_t c = next.fetch_add(1);
                if (c >= nchunks) break;
                int64_t a = c * chunk, b = std::min(n, a + chunk);
                f(a, b, t);
            }
        });
    for (auto &x : th) x.join();
}

static inline uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int draw_level(uint64_t seed, int64_t id, double ratio)
{
    uint64_t z = splitmix64(seed, (uint64_t)id);
    double u = ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    int l = (int)std::floor(-std::log(u) / std::log(ratio));
    return l > MAX_LEVEL ? MAX_LEVEL : l;
}

// k smallest of n indices by a SplitMix64 key: a seeded sample without replacement, sorted.
static std::vector<int64_t> sample(int64_t n, int64_t k, uint64_t seed)
{
    std::vector<int64_t> idx(n);
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    if (k >= n) return idx;
    std::vector<uint64_t> key(n);
    for (int64_t i = 0; i < n; i++) key[i] = splitmix64(seed, (uint64_t)i);
    std::nth_element(idx.begin(), idx.begin() + k, idx.end(),
                     [&](int64_t a, int64_t b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    idx.resize(k);
    std::sort(idx.begin(), idx.end());
    return idx;
}

void splits(int d, int M, std::vector<int> &off, std::vector<int> &len)
{
    off.resize(M);
    len.resize(M);
    int base = d / M, extra = d % M, o = 0;
    for (int j = 0; j < M; j++) {
        len[j] = base + (j < extra ? 1 : 0);
        off[j] = o;
        o += len[j];
    }
}

static inline float l2f(const float *a, const float *b, int d)
{
    float s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
    int t = 0;
    for (; t + 8 <= d; t += 8) {
        float x0 = a[t] - b[t], x1 = a[t + 1] - b[t + 1], x2 = a[t + 2] - b[t + 2], x3 = a[t + 3] - b[t + 3];
        float x4 = a[t + 4] - b[t + 4], x5 = a[t + 5] - b[t + 5], x6 = a[t + 6] - b[t + 6], x7 = a[t + 7] - b[t + 7];
        s0 += x0 * x0; s1 += x1 * x1; s2 += x2 * x2; s3 += x3 * x3;
        s4 += x4 * x4; s5 += x5 * x5; s6 += x6 * x6; s7 += x7 * x7;
    }
    for (; t < d; t++) {
        float x = a[t] - b[t];
        s0 += x * x;
    }
    return ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7));
}

// ------------------------------------------------------------------------------------------
// k-means (Lloyd).  Initial centres: a seeded sample of the points without replacement;
// ties go to the lowest centre index; an empty cluster is re-seeded with the point of the
// largest cluster furthest from its centre.  Points are rows of X at the given stride,
// coordinates [0, dim).
// dev, when given, runs the assignment step elsewhere (the device) with the same arithmetic:
// dev(C, cn, as, dm) fills as / dm for centres C [K][dim] with squared norms cn, or returns
// false (the step then runs here).
template <class T>
static void kmeans(const T *X, int64_t n, int64_t stride, int dim, int K, int iters,
                   uint64_t seed, T *C, bool have_init, int nt,
                   const std::function<bool(const T *, const T *, int32_t *, double *)> &dev = nullptr)
{
    if (!have_init) {
        if (n >= K) {
            auto pick = sample(n, K, seed);
            for (int c = 0; c < K; c++)
                for (int t = 0; t < dim; t++) C[(int64_t)c * dim + t] = X[pick[c] * stride + t];
        } else {
            for (int c = 0; c < K; c++) {
                int64_t i = (int64_t)(splitmix64(seed, c) % (uint64_t)n);
                for (int t = 0; t < dim; t++) C[(int64_t)c * dim + t] = X[i * stride + t];
            }
        }
    }
    std::vector<int32_t> as(n);
    std::vector<double> dm(n);
    std::vector<T> CT((size_t)dim * K), cn(K);
    for (int it = 0; it < iters; it++) {
        // assignment by ||c||^2 - 2 x.c over centres laid out [dim][K] (vectorises over c);
        // the exact distance of the chosen centre is recomputed for the empty-cluster rule
        for (int c = 0; c < K; c++) {
            T s = 0;
            for (int t = 0; t < dim; t++) {
                CT[(size_t)t * K + c] = C[(int64_t)c * dim + t];
                s += C[(int64_t)c * dim + t] * C[(int64_t)c * dim + t];
            }
            cn[c] = s;
        }
        if (!(dev && dev(C, cn.data(), as.data(), dm.data())))
        parallel_for(n, nt, 2048, [&](int64_t a, int64_t b, int) {
            std::vector<T> acc(K);
            for (int64_t i = a; i < b; i++) {
                const T *x = X + i * stride;
                for (int c = 0; c < K; c++) acc[c] = cn[c];
                for (int t = 0; t < dim; t++) {
                    T m2x = (T)-2 * x[t];
                    const T *ct = CT.data() + (size_t)t * K;
                    for (int c = 0; c < K; c++) acc[c] += m2x * ct[c];
                }
                int best = 0;
                for (int c = 1; c < K; c++)
                    if (acc[c] < acc[best]) best = c;
                as[i] = best;
                double s = 0;
                for (int t = 0; t < dim; t++) {
                    double df = (double)x[t] - (double)C[(int64_t)best * dim + t];
                    s += df * df;
                }
                dm[i] = s;
            }
        });
        std::vector<double> sums((size_t)K * dim, 0.0);
        std::vector<int64_t> cnt(K, 0);
        for (int64_t i = 0; i < n; i++) {
            int c = as[i];
            cnt[c]++;
            const T *x = X + i * stride;
            for (int t = 0; t < dim; t++) sums[(size_t)c * dim + t] += (double)x[t];
        }
        for (int c = 0; c < K; c++)
            if (cnt[c] > 0)
                for (int t = 0; t < dim; t++) C[(int64_t)c * dim + t] = (T)(sums[(size_t)c * dim + t] / cnt[c]);
        for (int c = 0; c < K; c++) {
            if (cnt[c] > 0) continue;
            int big = (int)(std::max_element(cnt.begin(), cnt.end()) - cnt.begin());
            if (cnt[big] < 2) continue;
            int64_t far = -1;
            for (int64_t i = 0; i < n; i++)
                if (as[i] == big && (far < 0 || dm[i] > dm[far])) far = i;
            for (int t = 0; t < dim; t++) C[(int64_t)c * dim + t] = X[far * stride + t];
            as[far] = c;
            cnt[big]--;
            cnt[c] = 1;
            dm[far] = 0;
        }
    }
}

static void pq_train(const float *Xall, int64_t nall, int d, int M, int iters, uint64_t seed,
                     float *C, bool have_init, int nt)
{
    std::vector<int> off, len;
    splits(d, M, off, len);
    // at most 256 training points per centroid (a seeded subset)
    const int64_t cap = (int64_t)KSUB * 256;
    std::vector<float> sub;
    const float *X = Xall;
    int64_t n = nall;
    if (nall > cap) {
        auto pick = sample(nall, cap, seed ^ 0x5bd1e995ULL);
        sub.resize((size_t)cap * d);
        for (int64_t i = 0; i < cap; i++) std::memcpy(sub.data() + i * d, Xall + pick[i] * d, sizeof(float) * d);
        X = sub.data();
        n = cap;
    }
    for (int j = 0; j < M; j++) {
        int o = off[j], l = len[j];
        std::vector<float> Cj((size_t)KSUB * l);
        if (have_init)
            for (int c = 0; c < KSUB; c++)
                for (int t = 0; t < l; t++) Cj[(size_t)c * l + t] = C[(int64_t)c * d + o + t];
        kmeans<float>(X + o, n, d, l, KSUB, iters, seed + 1000003ULL * (uint64_t)j, Cj.data(),
                      have_init, nt);
        for (int c = 0; c < KSUB; c++)
            for (int t = 0; t < l; t++) C[(int64_t)c * d + o + t] = Cj[(size_t)c * l + t];
    }
}

static void pq_encode(const float *X, int64_t n, int d, int M, const float *C, uint8_t *codes,
                      int nt)
{
    std::vector<int> off, len;
    splits(d, M, off, len);
    // per sub-space: centroids transposed [len][256] and their squared norms
    std::vector<std::vector<float>> CT(M), cn(M);
    for (int j = 0; j < M; j++) {
        CT[j].resize((size_t)len[j] * KSUB);
        cn[j].assign(KSUB, 0.f);
        for (int c = 0; c < KSUB; c++)
            for (int t = 0; t < len[j]; t++) {
                float v = C[(int64_t)c * d + off[j] + t];
                CT[j][(size_t)t * KSUB + c] = v;
                cn[j][c] += v * v;
            }
    }
    parallel_for(n, nt, 2048, [&](int64_t a, int64_t b, int) {
        float acc[KSUB];
        for (int64_t i = a; i < b; i++) {
            const float *x = X + i * d;
            for (int j = 0; j < M; j++) {
                for (int c = 0; c < KSUB; c++) acc[c] = cn[j][c];
                for (int t = 0; t < len[j]; t++) {
                    float m2x = -2.f * x[off[j] + t];
                    const float *ct = CT[j].data() + (size_t)t * KSUB;
                    for (int c = 0; c < KSUB; c++) acc[c] += m2x * ct[c];
                }
                int best = 0;
                for (int c = 1; c < KSUB; c++)
                    if (acc[c] < acc[best]) best = c;
                codes[i * M + j] = (uint8_t)best;
            }
        }
    });
}

// out[i] = decode(codes[i]) (+ out[i] if accumulate)
static void pq_decode(const uint8_t *codes, int64_t n, int d, int M, const float *C, float *out,
                      bool accumulate, int nt)
{
    std::vector<int> off, len;
    splits(d, M, off, len);
    parallel_for(n, nt, 8192, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; i++)
            for (int j = 0; j < M; j++) {
                const float *cc = C + (int64_t)codes[i * M + j] * d + off[j];
                float *o = out + i * d + off[j];
                for (int t = 0; t < len[j]; t++) o[t] = accumulate ? o[t] + cc[t] : cc[t];
            }
    });
}

// Y = X R^T, rows of length d (axpy form: vectorises over the output coordinate).
static void rotate(const float *X, int64_t n, int d, const float *R, float *Y, int nt)
{
    std::vector<float> RT((size_t)d * d);
    for (int t = 0; t < d; t++)
        for (int u = 0; u < d; u++) RT[(size_t)u * d + t] = R[(size_t)t * d + u];
    parallel_for(n, nt, 1024, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; i++) {
            float *y = Y + i * d;
            for (int t = 0; t < d; t++) y[t] = 0.f;
            for (int u = 0; u < d; u++) {
                float xu = X[i * d + u];
                const float *r = RT.data() + (size_t)u * d;
                for (int t = 0; t < d; t++) y[t] += r[t] * xu;
            }
        }
    });
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (destroyed):
// A = V diag(w) V^T, V column-major by eigenvector (V[r*n + c] = component r of vector c).
static void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &V, std::vector<double> &w)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0, tot = 0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) {
                double v = A[(size_t)p * n + q] * A[(size_t)p * n + q];
                tot += v;
                if (p != q) off += v;
            }
        if (off <= 1e-30 * tot || off == 0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
                double c = 1 / std::sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < n; k++) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; i++) w[i] = A[(size_t)i * n + i];
}

// Orthogonal polar factor of M (d x d, row-major): R = M (M^T M)^{-1/2} = U V^T, then
// re-orthonormalised by modified Gram-Schmidt on the rows.
static void polar(const std::vector<double> &M, int d, float *R)
{
    std::vector<double> S((size_t)d * d, 0.0);
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) {
            double s = 0;
            for (int k = 0; k < d; k++) s += M[(size_t)k * d + i] * M[(size_t)k * d + j];
            S[(size_t)i * d + j] = s;
        }
    std::vector<double> V, w;
    jacobi_eigen(d, S, V, w);
    double wmax = *std::max_element(w.begin(), w.end());
    std::vector<double> Sinv((size_t)d * d, 0.0);   // V diag(w^-1/2) V^T
    for (int k = 0; k < d; k++) {
        double f = w[k] > 1e-14 * wmax ? 1.0 / std::sqrt(w[k]) : 0.0;
        for (int i = 0; i < d; i++)
            for (int j = 0; j < d; j++) Sinv[(size_t)i * d + j] += V[(size_t)i * d + k] * f * V[(size_t)j * d + k];
    }
    std::vector<double> Rd((size_t)d * d, 0.0);
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) {
            double s = 0;
            for (int k = 0; k < d; k++) s += M[(size_t)i * d + k] * Sinv[(size_t)k * d + j];
            Rd[(size_t)i * d + j] = s;
        }
    for (int i = 0; i < d; i++) {
        for (int p = 0; p < i; p++) {
            double dot = 0;
            for (int k = 0; k < d; k++) dot += Rd[(size_t)i * d + k] * Rd[(size_t)p * d + k];
            for (int k = 0; k < d; k++) Rd[(size_t)i * d + k] -= dot * Rd[(size_t)p * d + k];
        }
        double nr = 0;
        for (int k = 0; k < d; k++) nr += Rd[(size_t)i * d + k] * Rd[(size_t)i * d + k];
        nr = std::sqrt(nr);
        for (int k = 0; k < d; k++) Rd[(size_t)i * d + k] = nr > 0 ? Rd[(size_t)i * d + k] / nr : (k == i);
    }
    for (size_t i = 0; i < (size_t)d * d; i++) R[i] = (float)Rd[i];
}

lc_status build_train(lc_index *ix, const float *xt, int64_t nt_)
{
    const lc_params &p = ix->p;
    int d = p.d, nt = n_threads(p);
    ix->R.assign((size_t)d * d, 0.f);
    for (int i = 0; i < d; i++) ix->R[(size_t)i * d + i] = 1.f;
    ix->C1.assign((size_t)KSUB * d, 0.f);
    ix->C2.assign((size_t)KSUB * d, 0.f);
    std::vector<float> Xr((size_t)nt_ * d), dec((size_t)nt_ * d);
    std::vector<uint8_t> codes((size_t)nt_ * std::max(p.M1, p.M2));
    if (p.use_opq) {
        pq_train(xt, nt_, d, p.M1, 4, p.seed + 11, ix->C1.data(), false, nt);
        for (int it = 0; it < p.opq_iters; it++) {
            rotate(xt, nt_, d, ix->R.data(), Xr.data(), nt);
            pq_train(Xr.data(), nt_, d, p.M1, 1, p.seed + 11, ix->C1.data(), true, nt);
            pq_encode(Xr.data(), nt_, d, p.M1, ix->C1.data(), codes.data(), nt);
            pq_decode(codes.data(), nt_, d, p.M1, ix->C1.data(), dec.data(), false, nt);
            // M = sum_i xhat_i x_i^T; the rotation maximising tr(R^T M) is its polar factor.
            // Partial sums over fixed chunks of rows, added in chunk order: M (and so R and
            // the whole index) does not depend on the thread count or the scheduling.
            constexpr int64_t MCH = 4096;
            const int64_t nch = (nt_ + MCH - 1) / MCH;
            std::vector<std::vector<double>> part((size_t)nch);
            parallel_for(nch, nt, 1, [&](int64_t a, int64_t b, int) {
                for (int64_t ch = a; ch < b; ch++) {
                    auto &Mp = part[(size_t)ch];
                    Mp.assign((size_t)d * d, 0.0);
                    for (int64_t i = ch * MCH; i < std::min(nt_, (ch + 1) * MCH); i++)
                        for (int r = 0; r < d; r++) {
                            double y = dec[(size_t)i * d + r];
                            for (int c = 0; c < d; c++) Mp[(size_t)r * d + c] += y * (double)xt[i * d + c];
                        }
                }
            });
            std::vector<double> M((size_t)d * d, 0.0);
            for (auto &Mp : part)
                for (size_t k = 0; k < M.size(); k++) M[k] += Mp[k];
            polar(M, d, ix->R.data());
        }
        rotate(xt, nt_, d, ix->R.data(), Xr.data(), nt);
        pq_train(Xr.data(), nt_, d, p.M1, p.kmeans_iters, p.seed + 11, ix->C1.data(), true, nt);
    } else {
        std::memcpy(Xr.data(), xt, sizeof(float) * (size_t)nt_ * d);
        pq_train(Xr.data(), nt_, d, p.M1, p.kmeans_iters, p.seed + 11, ix->C1.data(), false, nt);
    }
    // level 2 on the level-1 residuals
    pq_encode(Xr.data(), nt_, d, p.M1, ix->C1.data(), codes.data(), nt);
    pq_decode(codes.data(), nt_, d, p.M1, ix->C1.data(), dec.data(), false, nt);
    for (size_t i = 0; i < Xr.size(); i++) Xr[i] -= dec[i];
    pq_train(Xr.data(), nt_, d, p.M2, p.kmeans_iters, p.seed + 500011, ix->C2.data(), false, nt);
    ix->trained = true;
    ix->dev_dirty = true;
    return LC_OK;
}

void decode_all(const lc_index *ix, std::vector<float> &xh)
{
    int d = ix->p.d, nt = n_threads(ix->p);
    xh.assign((size_t)ix->n * d, 0.f);
    pq_decode(ix->codes1.data(), ix->n, d, ix->p.M1, ix->C1.data(), xh.data(), false, nt);
    pq_decode(ix->codes2.data(), ix->n, d, ix->p.M2, ix->C2.data(), xh.data(), true, nt);
}

// ------------------------------------------------------------------------------------------
// Graph build
namespace {

using Key = std::pair<float, int32_t>;   // (distance, id), lexicographic

struct Graph {
    lc_index *ix;
    int d;
    const float *xh;

    int32_t *row(int l, int32_t v) {
        return l == 0 ? ix->adj0.data() + (int64_t)v * DEG
                      : ix->upper_adj.data() + (ix->upper_off[v] + l - 1) * DEG;
    }
    float *rowd(int l, int32_t v) {
        return l == 0 ? ix->adj0_d.data() + (int64_t)v * DEG
                      : ix->upper_d.data() + (ix->upper_off[v] + l - 1) * DEG;
    }
    int count(int l, int32_t v) {
        int32_t *r = row(l, v);
        int c = 0;
        while (c < DEG && r[c] >= 0) c++;
        return c;
    }
    float dist(int32_t a, int32_t b) const { return l2f(xh + (int64_t)a * d, xh + (int64_t)b * d, d); }
};

struct SearchState {
    std::vector<uint32_t> mark;
    uint32_t epoch = 0;
    std::vector<Key> W;

    void reset(int64_t n) {
        if ((int64_t)mark.size() < n) mark.assign(n, 0), epoch = 0;
        if (++epoch == 0) {
            std::fill(mark.begin(), mark.end(), 0);
            epoch = 1;
        }
    }
};

// Best-first search of level l from `entry` keeping the ef closest (result sorted by key).
static void search_layer(Graph &g, const float *x, int32_t entry, int ef, int l, SearchState &st)
{
    st.reset(g.ix->n);
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> C;   // min-heap
    std::priority_queue<Key> W;                                         // max-heap
    Key k0{l2f(x, g.xh + (int64_t)entry * g.d, g.d), entry};
    st.mark[entry] = st.epoch;
    C.push(k0);
    W.push(k0);
    while (!C.empty()) {
        Key c = C.top();
        C.pop();
        if (W.top() < c) break;
        const int32_t *r = g.row(l, c.second);
        for (int s = 0; s < DEG && r[s] >= 0; s++) {
            int32_t e = r[s];
            if (st.mark[e] == st.epoch) continue;
            st.mark[e] = st.epoch;
            Key ke{l2f(x, g.xh + (int64_t)e * g.d, g.d), e};
            if ((int)W.size() < ef || ke < W.top()) {
                C.push(ke);
                W.push(ke);
                if ((int)W.size() > ef) W.pop();
            }
        }
    }
    st.W.resize(W.size());
    for (int i = (int)W.size() - 1; i >= 0; i--) {
        st.W[i] = W.top();
        W.pop();
    }
}

// HNSW shrinking heuristic on candidates sorted by key w.r.t. the base point.
static int heuristic(Graph &g, const Key *cand, int n, int M, int32_t *out)
{
    int kept = 0;
    for (int s = 0; s < n && kept < M; s++) {
        bool good = true;
        for (int u = 0; u < kept; u++)
            if (g.dist(cand[s].second, out[u]) < cand[s].first) { good = false; break; }
        if (good) out[kept++] = cand[s].second;
    }
    return kept;
}

static void add_link(Graph &g, int l, int32_t owner, int32_t x)
{
    int32_t *id = g.row(l, owner);
    float *ds = g.rowd(l, owner);
    int n = g.count(l, owner);
    for (int s = 0; s < n; s++)
        if (id[s] == x) return;
    Key kx{g.dist(owner, x), x};
    Key cand[DEG + 1];
    int m = 0;
    bool ins = false;
    for (int s = 0; s < n; s++) {
        Key ks{ds[s], id[s]};
        if (!ins && kx < ks) { cand[m++] = kx; ins = true; }
        cand[m++] = ks;
    }
    if (!ins) cand[m++] = kx;
    if (m <= DEG) {
        for (int s = 0; s < m; s++) { id[s] = cand[s].second; ds[s] = cand[s].first; }
        return;
    }
    int32_t keep[DEG];
    int kn = heuristic(g, cand, m, DEG, keep);
    int s2 = 0;
    for (int s = 0; s < m && s2 < kn; s++)
        if (cand[s].second == keep[s2]) { id[s2] = cand[s].second; ds[s2] = cand[s].first; s2++; }
    for (int s = kn; s < DEG; s++) { id[s] = -1; ds[s] = 0.f; }
}

}  // namespace

// A back-link of an insertion batch: level, the node whose row receives it, the new node.
struct Link { int32_t level, target, src; };

// Orders the links by (level, target), keeping the order of equal keys (the batch lists them
// by increasing source): a stable least-significant-digit radix sort on 11-bit digits of
// (level << 32 | target).
static void sort_links(std::vector<Link> &links)
{
    const size_t n = links.size();
    if (n < 2) return;
    uint64_t top = 0;
    for (const Link &l : links) top = std::max(top, ((uint64_t)l.level << 32) | (uint32_t)l.target);
    std::vector<Link> tmp(n);
    constexpr int BITS = 11, NB = 1 << BITS;
    for (int shift = 0; shift < 64 && (top >> shift) != 0; shift += BITS) {
        size_t cnt[NB + 1] = {};
        auto digit = [&](const Link &l) {
            return (size_t)(((((uint64_t)l.level << 32) | (uint32_t)l.target) >> shift) & (NB - 1));
        };
        for (const Link &l : links) cnt[digit(l) + 1]++;
        for (int i = 0; i < NB; i++) cnt[i + 1] += cnt[i];
        for (const Link &l : links) tmp[cnt[digit(l)]++] = l;
        links.swap(tmp);
    }
}

static lc_status insert_range(lc_index *ix, const float *xr, int64_t first, int64_t count, int nt)
{
    const lc_params &p = ix->p;
    Graph g{ix, p.d, ix->xh.data()};
    std::vector<SearchState> states(nt);
    const bool gpu = p.build_gpu != 0;
    if (gpu) {
        lc_status rs = build_gpu_begin(ix);
        if (rs == LC_OK) rs = build_gpu_link0_begin(ix);
        if (rs != LC_OK) { build_gpu_end(ix); return rs; }
    }
    const int efc = p.ef_construction;
    std::vector<int64_t> gmem;                  // batch members searched on the device
    std::vector<int32_t> gslot, gsel;           // member -> row of the device selections
    std::vector<float> gxr;
    int64_t done = 0;
    while (done < count) {
        int64_t ncur = first + done;
        int64_t b = ncur / 16;
        if (b > p.batch_max) b = p.batch_max;
        if (b < 1) b = 1;
        if (ncur == 0) b = 1;
        if (done + b > count) b = count - done;
        int ml0 = ix->max_level;
        int32_t ep0 = ix->ep;
        // selections per batch member and level: sel[u][l] (up to DEG ids)
        std::vector<std::vector<int32_t>> sel(b);
        // level-0 members: their level-0 insertion searches run together on the device
        gmem.clear();
        gslot.assign(b, -1);
        if (gpu && ep0 >= 0) {
            for (int64_t u = 0; u < b; u++)
                if (ix->levels[ncur + u] == 0) { gslot[u] = (int32_t)gmem.size(); gmem.push_back(u); }
            const int64_t m = (int64_t)gmem.size();
            gxr.resize((size_t)m * p.d);
            for (int64_t i = 0; i < m; i++)
                std::memcpy(gxr.data() + i * p.d, xr + (ncur + gmem[i] - first) * p.d, sizeof(float) * p.d);
            gsel.resize((size_t)m * (DEG + 1));
            // queued on the device; the host searches of the higher-level members run meanwhile
            lc_status rs = build_gpu_select_start(ix, gxr.data(), m, efc, ep0, ml0);
            if (rs != LC_OK) { build_gpu_end(ix); return rs; }
        }
        parallel_for(b, nt, 8, [&](int64_t a, int64_t e, int t) {
            SearchState &st = states[t];
            for (int64_t u = a; u < e; u++) {
                int64_t x = ncur + u;
                const float *xv = xr + (x - first) * p.d;
                int Lx = ix->levels[x];
                int top = std::min(Lx, ml0);
                sel[u].assign((size_t)(top + 1) * (DEG + 1), -1);
                if (ep0 < 0) continue;
                if (gslot[u] >= 0) continue;       // level 0 searched and selected on the device
                int32_t cur = ep0;
                float dcur = l2f(xv, g.xh + (int64_t)cur * p.d, p.d);
                for (int l = ml0; l > Lx; l--) {
                    for (;;) {
                        const int32_t *r = g.row(l, cur);
                        Key best{0.f, -1};
                        for (int s = 0; s < DEG && r[s] >= 0; s++) {
                            Key ke{l2f(xv, g.xh + (int64_t)r[s] * p.d, p.d), r[s]};
                            if (best.second < 0 || ke < best) best = ke;
                        }
                        if (best.second >= 0 && best < Key{dcur, cur}) { cur = best.second; dcur = best.first; }
                        else break;
                    }
                }
                for (int l = top; l >= 0; l--) {
                    search_layer(g, xv, cur, p.ef_construction, l, st);
                    int32_t *out = sel[u].data() + (size_t)l * (DEG + 1);
                    out[DEG] = heuristic(g, st.W.data(), (int)st.W.size(), DEG, out);
                    cur = st.W[0].second;
                }
            }
        });
        if (gpu && ep0 >= 0) {
            lc_status rs = build_gpu_select_finish(ix, (int64_t)gmem.size(), gsel.data());
            if (rs != LC_OK) { build_gpu_end(ix); return rs; }
            for (int64_t u = 0; u < b; u++)
                if (gslot[u] >= 0)
                    std::memcpy(sel[u].data(), gsel.data() + (size_t)gslot[u] * (DEG + 1), sizeof(int32_t) * (DEG + 1));
        }
        // the new nodes' own rows, sorted by decoded-to-decoded distance (level 0 on the
        // device in the GPU-assisted build)
        const int l_own = gpu ? 1 : 0;
        parallel_for(b, nt, 64, [&](int64_t a, int64_t e, int) {
            for (int64_t u = a; u < e; u++) {
                int64_t x = ncur + u;
                int top = std::min((int)ix->levels[x], ml0);
                for (int l = l_own; l <= top && ep0 >= 0; l++) {
                    const int32_t *s = sel[u].data() + (size_t)l * (DEG + 1);
                    int cnt = s[DEG];
                    Key ks[DEG];
                    for (int i = 0; i < cnt; i++) ks[i] = Key{g.dist((int32_t)x, s[i]), s[i]};
                    std::sort(ks, ks + cnt);
                    int32_t *r = g.row(l, (int32_t)x);
                    float *rd = g.rowd(l, (int32_t)x);
                    for (int i = 0; i < cnt; i++) { r[i] = ks[i].second; rd[i] = ks[i].first; }
                }
            }
        });
        // back-links, grouped by (level, target); within a group in id order of the source
        std::vector<Link> links;
        for (int64_t u = 0; u < b; u++) {
            int64_t x = ncur + u;
            int top = std::min((int)ix->levels[x], ml0);
            for (int l = 0; l <= top && ep0 >= 0; l++) {
                const int32_t *s = sel[u].data() + (size_t)l * (DEG + 1);
                for (int i = 0; i < s[DEG]; i++) links.push_back({l, s[i], (int32_t)x});
            }
        }
        sort_links(links);
        std::vector<size_t> starts;
        for (size_t i = 0; i < links.size(); i++)
            if (i == 0 || links[i].level != links[i - 1].level || links[i].target != links[i - 1].target)
                starts.push_back(i);
        starts.push_back(links.size());
        // GPU-assisted build: level 0's own rows and back-links on the device (the groups of
        // level 0 come first), the upper levels here
        size_t g0 = 0;
        if (gpu)
            while (g0 + 1 < starts.size() && links[starts[g0]].level == 0) g0++;
        if (gpu && ep0 >= 0) {
            std::vector<int32_t> sel0((size_t)b * (DEG + 1));
            for (int64_t u = 0; u < b; u++) std::memcpy(sel0.data() + u * (DEG + 1), sel[u].data(), sizeof(int32_t) * (DEG + 1));
            std::vector<int32_t> tg(g0), st(g0 + 1), src(starts[g0]);
            for (size_t gi = 0; gi < g0; gi++) {
                tg[gi] = links[starts[gi]].target;
                st[gi] = (int32_t)starts[gi];
            }
            st[g0] = (int32_t)starts[g0];
            for (size_t i = 0; i < starts[g0]; i++) src[i] = links[i].src;
            lc_status rs = build_gpu_link0(ix, ncur, b, sel0.data(), tg.data(), st.data(), (int64_t)g0, src.data());
            if (rs != LC_OK) { build_gpu_end(ix); return rs; }
        }
        parallel_for((int64_t)(starts.size() - 1 - g0), nt, 64, [&](int64_t a, int64_t e, int) {
            for (int64_t gi = a + (int64_t)g0; gi < e + (int64_t)g0; gi++)
                for (size_t i = starts[gi]; i < starts[gi + 1]; i++)
                    add_link(g, links[i].level, links[i].target, links[i].src);
        });
        if (gpu) {
            // re-send the upper rows the batch wrote (level 0 was written on the device)
            std::vector<int64_t> rowsu;
            for (int64_t u = 0; u < b; u++) {
                int64_t x = ncur + u;
                for (int l = 1; l <= std::min((int)ix->levels[x], ml0); l++) rowsu.push_back(ix->upper_off[x] + l - 1);
            }
            for (size_t gi = g0; gi + 1 < starts.size(); gi++) {
                const Link &lk = links[starts[gi]];
                rowsu.push_back(ix->upper_off[lk.target] + lk.level - 1);
            }
            lc_status rs = build_gpu_rows(ix, nullptr, 0, rowsu.data(), (int64_t)rowsu.size());
            if (rs != LC_OK) { build_gpu_end(ix); return rs; }
        }
        for (int64_t u = 0; u < b; u++) {
            int64_t x = ncur + u;
            if (ix->levels[x] > ix->max_level) { ix->max_level = ix->levels[x]; ix->ep = (int32_t)x; }
        }
        done += b;
    }
    if (gpu) {
        lc_status rs = build_gpu_link0_end(ix);
        build_gpu_end(ix);
        if (rs != LC_OK) return rs;
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------------------
// Regression codebook
namespace {

struct NormalEq {
    double A[45];   // upper triangle of G G^T (9 x 9), row-major packed
    double b[9];    // G x
    double xx;      // ||x||^2
};

static inline int tri(int i, int j) { return i <= j ? i * 9 - i * (i - 1) / 2 + (j - i) : tri(j, i); }

// Normal equations of vector i over the coordinates [t0, t1) (one regression block).
static void normal_eq(const lc_index *ix, int64_t i, const float *x, int t0, int t1, NormalEq &ne)
{
    int d = ix->p.d;
    const float *G[9];
    G[0] = ix->xh.data() + i * d;
    for (int j = 1; j <= KBETA; j++) {
        int32_t v = ix->adj0[i * DEG + j - 1];
        G[j] = v >= 0 ? ix->xh.data() + (int64_t)v * d : nullptr;
    }
    for (int a = 0; a < 9; a++) {
        double s = 0;
        if (G[a])
            for (int t = t0; t < t1; t++) s += (double)G[a][t] * x[t];
        ne.b[a] = s;
        for (int c = a; c < 9; c++) {
            double u = 0;
            if (G[a] && G[c])
                for (int t = t0; t < t1; t++) u += (double)G[a][t] * G[c][t];
            ne.A[tri(a, c)] = u;
        }
    }
    double xx = 0;
    for (int t = t0; t < t1; t++) xx += (double)x[t] * x[t];
    ne.xx = xx;
}

// Solves (A + lambda I) beta = b, lambda = 1e-10 trace(A) / 9 (increased if needed).
static void ridge_solve(const double *Ap, const double *b, double *beta)
{
    double tr = 0;
    for (int i = 0; i < 9; i++) tr += Ap[tri(i, i)];
    double lam = tr > 0 ? 1e-10 * tr / 9 : 1e-300;
    for (int attempt = 0; attempt < 8; attempt++, lam *= 100) {
        double L[9][9] = {};
        bool ok = true;
        for (int i = 0; i < 9 && ok; i++)
            for (int j = 0; j <= i; j++) {
                double s = Ap[tri(i, j)] + (i == j ? lam : 0.0);
                for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k];
                if (i == j) {
                    if (s <= 0) { ok = false; break; }
                    L[i][i] = std::sqrt(s);
                } else {
                    L[i][j] = s / L[j][j];
                }
            }
        if (!ok) continue;
        double y[9];
        for (int i = 0; i < 9; i++) {
            double s = b[i];
            for (int k = 0; k < i; k++) s -= L[i][k] * y[k];
            y[i] = s / L[i][i];
        }
        for (int i = 8; i >= 0; i--) {
            double s = y[i];
            for (int k = i + 1; k < 9; k++) s -= L[k][i] * beta[k];
            beta[i] = s / L[i][i];
        }
        return;
    }
    for (int i = 0; i < 9; i++) beta[i] = i == 0 ? 1.0 : 0.0;
}

// ||x - beta^T G||^2 = ||x||^2 - 2 beta.b + beta^T A beta
static inline double quad_loss(const NormalEq &ne, const double *beta)
{
    double s = ne.xx;
    for (int i = 0; i < 9; i++) {
        s -= 2 * beta[i] * ne.b[i];
        s += beta[i] * beta[i] * ne.A[tri(i, i)];
        for (int j = i + 1; j < 9; j++) s += 2 * beta[i] * beta[j] * ne.A[tri(i, j)];
    }
    return s;
}

// argmin over the K codewords Bd [K][9] (ties to the lowest index)
static int argmin_codeword(const NormalEq &ne, const double *Bd, int K)
{
    int best = 0;
    double bl = INFINITY;
    for (int c = 0; c < K; c++) {
        double l = quad_loss(ne, Bd + c * 9);
        if (l < bl) { bl = l; best = c; }
    }
    return best;
}

}  // namespace

// Regression codebooks (Section 4.3), one per block of coordinates (the product codebook;
// one block = the plain codebook): trained on a seeded subset of the vectors just added.
// beta_K > 1: k-means of the per-vector least-squares weights initialises codewords
// 1..K-1 (codeword 0 stays e0), then EM alternates argmin assignment and per-cluster least
// squares.  beta_K = 1: the shared least-squares weights beta* of Section 4.2 per block.
static lc_status train_codebook(lc_index *ix, const float *xr, int64_t first, int64_t count, int nt)
{
    const lc_params &p = ix->p;
    const int bM = p.beta_M, bK = p.beta_K;
    std::vector<int> off, len;
    splits(p.d, bM, off, len);
    auto sub = sample(count, std::min<int64_t>(count, p.beta_train_n), p.seed + 5);
    int64_t ns = (int64_t)sub.size();
    std::vector<NormalEq> ne(ns);
    std::vector<double> per((size_t)ns * 9);
    std::vector<double> Ball((size_t)bM * bK * 9, 0.0);
    for (int m = 0; m < bM; m++) {
        const int t0 = off[m], t1 = off[m] + len[m];
        parallel_for(ns, nt, 1024, [&](int64_t a, int64_t b, int) {
            for (int64_t s = a; s < b; s++) {
                int64_t i = sub[s];
                normal_eq(ix, first + i, xr + i * p.d, t0, t1, ne[s]);
                if (bK > 1) ridge_solve(ne[s].A, ne[s].b, per.data() + s * 9);
            }
        });
        double *Bd = Ball.data() + (size_t)m * bK * 9;
        if (bK == 1) {
            double SA[45] = {}, Sb[9] = {};
            for (int64_t s = 0; s < ns; s++) {
                for (int k = 0; k < 45; k++) SA[k] += ne[s].A[k];
                for (int k = 0; k < 9; k++) Sb[k] += ne[s].b[k];
            }
            ridge_solve(SA, Sb, Bd);
            continue;
        }
        for (int c = 0; c < bK; c++) Bd[(size_t)c * 9] = 1.0;          // e0 everywhere to start
        int K = (int)std::min<int64_t>(bK - 1, ns);
        // GPU-assisted build: the assignment steps of the k-means and of the EM on the device
        // (the same arithmetic; the sums stay here, in the same order)
        EmDev *em = nullptr;
        if (p.build_gpu) {
            std::vector<double> ne55((size_t)ns * 55);
            for (int64_t s = 0; s < ns; s++) {
                std::memcpy(ne55.data() + s * 55, ne[s].A, sizeof(double) * 45);
                std::memcpy(ne55.data() + s * 55 + 45, ne[s].b, sizeof(double) * 9);
                ne55[s * 55 + 54] = ne[s].xx;
            }
            em = em_begin(per.data(), ns, 9, ne55.data());
            if (!em) {
                set_error("device memory for the regression-codebook training failed: %s",
                          cudaGetErrorString(cudaGetLastError()));
                return LC_ERR_CUDA;
            }
        }
        bool dev_ok = true;
        std::function<bool(const double *, const double *, int32_t *, double *)> dev_nearest;
        if (em)
            dev_nearest = [&](const double *C, const double *cn, int32_t *a, double *dmv) {
                return dev_ok = dev_ok && em_nearest(em, C, cn, K, a, dmv);
            };
        if (K > 0)
            kmeans<double>(per.data(), ns, 9, 9, K, 25, p.seed + 31 + 101 * (uint64_t)m, Bd + 9, false, nt, dev_nearest);
        std::vector<int32_t> as(ns);
        for (int it = 0; it < p.beta_iters; it++) {
            if (em) {
                dev_ok = dev_ok && em_assign(em, Bd, bK, as.data());
            } else {
                parallel_for(ns, nt, 2048, [&](int64_t a, int64_t b, int) {
                    for (int64_t s = a; s < b; s++) as[s] = argmin_codeword(ne[s], Bd, bK);
                });
            }
            if (!dev_ok) {
                em_free(em);
                set_error("regression-codebook training on the device failed");
                return LC_ERR_CUDA;
            }
            std::vector<double> SA((size_t)bK * 45, 0.0), Sb((size_t)bK * 9, 0.0);
            std::vector<int64_t> cnt(bK, 0);
            for (int64_t s = 0; s < ns; s++) {
                int c = as[s];
                cnt[c]++;
                for (int k = 0; k < 45; k++) SA[(size_t)c * 45 + k] += ne[s].A[k];
                for (int k = 0; k < 9; k++) Sb[(size_t)c * 9 + k] += ne[s].b[k];
            }
            for (int c = 1; c < bK; c++)
                if (cnt[c] > 0) ridge_solve(SA.data() + (size_t)c * 45, Sb.data() + (size_t)c * 9, Bd + (size_t)c * 9);
        }
        em_free(em);
        if (!dev_ok) {
            set_error("regression-codebook training on the device failed");
            return LC_ERR_CUDA;
        }
    }
    ix->B.resize(Ball.size());
    for (size_t k = 0; k < ix->B.size(); k++) ix->B[k] = (float)Ball[k];
    ix->has_codebook = true;
    return LC_OK;
}

// Each vector's codeword per block: argmin of the block's loss under the index's codebooks.
static void assign_codewords(lc_index *ix, const float *xr, int64_t first, int64_t count, int nt)
{
    const int bM = ix->p.beta_M, bK = ix->p.beta_K;
    if (bK == 1) {
        std::fill(ix->beta.begin() + first * bM, ix->beta.begin() + (first + count) * bM, 0);
        return;
    }
    std::vector<int> off, len;
    splits(ix->p.d, bM, off, len);
    std::vector<double> Bd(ix->B.begin(), ix->B.end());
    parallel_for(count, nt, 1024, [&](int64_t a, int64_t b, int) {
        NormalEq ne;
        for (int64_t i = a; i < b; i++)
            for (int m = 0; m < bM; m++) {
                normal_eq(ix, first + i, xr + i * ix->p.d, off[m], off[m] + len[m], ne);
                ix->beta[(first + i) * bM + m] = (uint8_t)argmin_codeword(ne, Bd.data() + (size_t)m * bK * 9, bK);
            }
    });
}

// Rebuilds the build-side state (decoded vectors, row distances) of an index that was
// imported or loaded, so that more vectors can be added.
static void ensure_build_state(lc_index *ix)
{
    int64_t n = ix->n;
    if ((int64_t)ix->xh.size() == n * ix->p.d && (int64_t)ix->adj0_d.size() == n * DEG) return;
    decode_all(ix, ix->xh);
    Graph g{ix, ix->p.d, ix->xh.data()};
    ix->adj0_d.assign((size_t)n * DEG, 0.f);
    for (int64_t i = 0; i < n; i++)
        for (int s = 0; s < DEG && ix->adj0[i * DEG + s] >= 0; s++)
            ix->adj0_d[i * DEG + s] = g.dist((int32_t)i, ix->adj0[i * DEG + s]);
    ix->upper_d.assign(ix->upper_adj.size(), 0.f);
    for (int64_t i = 0; i < n; i++)
        for (int l = 1; l <= ix->levels[i]; l++)
            for (int s = 0; s < DEG; s++) {
                int32_t v = g.row(l, (int32_t)i)[s];
                if (v >= 0) g.rowd(l, (int32_t)i)[s] = g.dist((int32_t)i, v);
            }
}

lc_status build_add(lc_index *ix, const float *x, int64_t n)
{
    const lc_params &p = ix->p;
    int d = p.d, nt = n_threads(p);
    if (p.build_gpu) {
        // checked before the index is touched: a failed add leaves it as it was
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            set_error("build_gpu = 1 needs a CUDA device");
            return LC_ERR_CUDA;
        }
    }
    ensure_build_state(ix);
    int64_t first = ix->n, total = first + n;
    std::vector<float> xr((size_t)n * d);
    std::vector<uint8_t> nc1((size_t)n * p.M1), nc2((size_t)n * p.M2);
    if (p.build_gpu) {
        // rotation and both code levels on the device (the host's arithmetic, the host's codes)
        lc_status rs = build_gpu_encode(ix, x, n, xr.data(), nc1.data(), nc2.data());
        if (rs != LC_OK) return rs;
    } else {
        rotate(x, n, d, ix->R.data(), xr.data(), nt);
        std::vector<float> xh1((size_t)n * d);
        pq_encode(xr.data(), n, d, p.M1, ix->C1.data(), nc1.data(), nt);
        pq_decode(nc1.data(), n, d, p.M1, ix->C1.data(), xh1.data(), false, nt);
        for (size_t i = 0; i < xh1.size(); i++) xh1[i] = xr[i] - xh1[i];       // the residual
        pq_encode(xh1.data(), n, d, p.M2, ix->C2.data(), nc2.data(), nt);
    }
    ix->codes1.resize((size_t)total * p.M1);
    ix->codes2.resize((size_t)total * p.M2);
    ix->beta.resize((size_t)total * p.beta_M, 0);
    ix->xh.resize((size_t)total * d);
    uint8_t *c1 = ix->codes1.data() + first * p.M1;
    uint8_t *c2 = ix->codes2.data() + first * p.M2;
    float *xh = ix->xh.data() + first * d;
    std::memcpy(c1, nc1.data(), nc1.size());
    std::memcpy(c2, nc2.data(), nc2.size());
    pq_decode(c1, n, d, p.M1, ix->C1.data(), xh, false, nt);
    pq_decode(c2, n, d, p.M2, ix->C2.data(), xh, true, nt);
    // levels and row storage
    ix->levels.resize(total);
    ix->upper_off.resize(total, -1);
    int64_t rows = (int64_t)ix->upper_adj.size() / DEG;
    for (int64_t i = first; i < total; i++) {
        int L = draw_level(p.seed, i, (double)p.level_ratio);
        ix->levels[i] = L;
        ix->upper_off[i] = L > 0 ? rows : -1;
        rows += L;
    }
    ix->upper_adj.resize((size_t)rows * DEG, -1);
    ix->upper_d.resize((size_t)rows * DEG, 0.f);
    ix->adj0.resize((size_t)total * DEG, -1);
    ix->adj0_d.resize((size_t)total * DEG, 0.f);
    ix->n = total;
    lc_status rs = insert_range(ix, xr.data(), first, n, nt);
    if (rs != LC_OK) return rs;
    if (!ix->has_codebook) {
        rs = train_codebook(ix, xr.data(), first, n, nt);
        if (rs != LC_OK) return rs;
    }
    if (p.build_gpu) {
        rs = build_gpu_assign(ix, xr.data(), first, n);
        if (rs != LC_OK) return rs;
    } else {
        assign_codewords(ix, xr.data(), first, n, nt);
    }
    ix->dev_dirty = true;
    return LC_OK;
}

}  // namespace lc
