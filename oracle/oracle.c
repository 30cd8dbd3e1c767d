/*
 * FP64 CPU oracle for the neighbourhood-graph step (exact kNN followed by
 * UMAP-style fuzzy connectivities).  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the library under
 * test never does.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes, and the passage each part follows:
 *   - Distances (paper, Methods, "Custom GPU kernels"): squared Euclidean
 *     ||x_i - x_j||^2 and cosine 1 - x_i.x_j / (|x_i| |x_j|).  The graph uses
 *     the metric (non-squared) Euclidean distance, as scanpy's neighbours
 *     step does (paper, "Implementation": functions follow scanpy).
 *   - kNN: brute force, every pair by direct difference in double, sorted by
 *     (distance, index) ascending; the first k kept, self included.
 *   - rho_i: the smallest non-zero distance of row i (local connectivity 1).
 *   - sigma_i: bisection on sum_{c>=1} exp(-max(0, d_ic - rho_i) / sigma)
 *     = log2(k) (column 0, the self slot, skipped), at most 64 steps, stop
 *     when within 1e-5 of the target; floor 1e-3 * mean row distance (rho>0)
 *     or 1e-3 * mean of all distances (rho == 0).
 *   - directed weight w_ic: 0 for the row itself, 1 when d <= rho or
 *     sigma == 0, else exp(-(d - rho) / sigma).
 *   - G = A + A^T - A o A^T, diagonal and zeros dropped, CSR with ascending
 *     columns.
 * The paper states the graph is stored for UMAP/Leiden (Methods, "Dimensionality
 * reduction and graph analysis"); the rho/sigma/union definitions are those of
 * the UMAP method that scanpy follows.
 *   - UMAP layout (same passage; the UMAP method's embedding optimisation):
 *     edge-sampled SGD on the graph, epoch by epoch, with its readings stated
 *     above oracle_umap_epochs; negative samples from SplitMix64.
 *   - E-distance (Methods, "Perturbation distance computation"): sums of
 *     Euclidean distances per group pair by direct difference, means, and
 *     E = 2 d_ab - d_aa - d_bb.
 *   - Approximate kNN by NN-descent (the paper's CPU neighbour search is
 *     PyNNDescent, Methods, "Benchmarking"; the method is Dong, Charikar & Li,
 *     WWW 2011): the synchronous variant stated above oracle_nndescent.  Its
 *     list decisions are taken on FP32 squared distances (sequential fused
 *     multiply-adds), the precision the GPU decides in, so that both sides
 *     take the same integer decisions.
 *
 * All arithmetic is double; inputs are the float32 arrays the GPU reads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_BAD_ARG 1
#define ORC_NO_MEM 2
#define ORC_CAPACITY 3

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Distance between rows a and b of length d; metric 0 = Euclidean (metric,
 * not squared), 1 = cosine distance on the given rows (1 - cos). */
static double pair_distance(const float *a, const float *b, int d, int metric) {
    if (metric == 0) {
        double s = 0.0;
        for (int t = 0; t < d; ++t) {
            double diff = (double)a[t] - (double)b[t];
            s += diff * diff;
        }
        return sqrt(s);
    } else {
        double ab = 0.0, aa = 0.0, bb = 0.0;
        for (int t = 0; t < d; ++t) {
            ab += (double)a[t] * (double)b[t];
            aa += (double)a[t] * (double)a[t];
            bb += (double)b[t] * (double)b[t];
        }
        /* all-zero rows: distance 0 between two of them, 1 to any other row */
        if (aa == 0.0 && bb == 0.0) return 0.0;
        if (aa == 0.0 || bb == 0.0) return 1.0;
        return 1.0 - ab / (sqrt(aa) * sqrt(bb));
    }
}

/* (d, j) < (d', j') in the (distance, index) order. */
static int before(double d, int64_t j, double d2, int64_t j2) {
    return d < d2 || (d == d2 && j < j2);
}

/*
 * Exact kNN for nq query rows (ids in `queries`, or all rows 0..n-1 when
 * queries == NULL) against all n rows of X (row-major n x d float32).
 * Outputs: idx [nq, k] int32, dist [nq, k] double ascending, next [nq] the
 * (k+1)-th distance (INFINITY when k == n), used to judge boundary ties.
 */
int oracle_knn(const float *X, int64_t n, int d, const int64_t *queries, int64_t nq,
               int k, int metric, int32_t *idx, double *dist, double *next) {
    if (!X || n <= 0 || d <= 0 || k <= 0 || k > n || nq < 0 || (metric != 0 && metric != 1))
        return ORC_BAD_ARG;
    int kk = (k < n) ? k + 1 : k;      /* keep one extra for `next` */
    int bad = 0;
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)kk);
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)kk);
        if (!bd || !bj) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t qi = 0; qi < nq; ++qi) {
                int64_t i = queries ? queries[qi] : qi;
                const float *xi = X + (size_t)i * (size_t)d;
                int cnt = 0;
                for (int64_t j = 0; j < n; ++j) {
                    double dj = pair_distance(xi, X + (size_t)j * (size_t)d, d, metric);
                    if (cnt == kk && !before(dj, j, bd[kk - 1], bj[kk - 1])) continue;
                    /* insertion into the sorted prefix */
                    int p = (cnt < kk) ? cnt++ : kk - 1;
                    while (p > 0 && before(dj, j, bd[p - 1], bj[p - 1])) {
                        bd[p] = bd[p - 1];
                        bj[p] = bj[p - 1];
                        --p;
                    }
                    bd[p] = dj;
                    bj[p] = j;
                }
                for (int c = 0; c < k; ++c) {
                    idx[(size_t)qi * k + c] = (int32_t)bj[c];
                    dist[(size_t)qi * k + c] = bd[c];
                }
                if (next) next[qi] = (kk > k) ? bd[k] : INFINITY;
            }
        }
        free(bd);
        free(bj);
    }
    return bad ? ORC_NO_MEM : ORC_OK;
}

/*
 * Exact kNN of nq external query rows Q against the nd rows of D (both
 * row-major float32 with d columns); ids index D.  Same order and tie rule
 * as oracle_knn.  Used for neighbours restricted to one sample of a batch.
 */
int oracle_knn_qd(const float *Q, int64_t nq, const float *D, int64_t nd, int d, int k, int metric,
                  int32_t *idx, double *dist, double *next) {
    if (!Q || !D || nq < 0 || nd <= 0 || d <= 0 || k <= 0 || k > nd || (metric != 0 && metric != 1))
        return ORC_BAD_ARG;
    int kk = (k < nd) ? k + 1 : k;
    int bad = 0;
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)kk);
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)kk);
        if (!bd || !bj) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t qi = 0; qi < nq; ++qi) {
                const float *xi = Q + (size_t)qi * (size_t)d;
                int cnt = 0;
                for (int64_t j = 0; j < nd; ++j) {
                    double dj = pair_distance(xi, D + (size_t)j * (size_t)d, d, metric);
                    if (cnt == kk && !before(dj, j, bd[kk - 1], bj[kk - 1])) continue;
                    int p = (cnt < kk) ? cnt++ : kk - 1;
                    while (p > 0 && before(dj, j, bd[p - 1], bj[p - 1])) {
                        bd[p] = bd[p - 1];
                        bj[p] = bj[p - 1];
                        --p;
                    }
                    bd[p] = dj;
                    bj[p] = j;
                }
                for (int c = 0; c < k; ++c) {
                    idx[(size_t)qi * k + c] = (int32_t)bj[c];
                    dist[(size_t)qi * k + c] = bd[c];
                }
                if (next) next[qi] = (kk > k) ? bd[k] : INFINITY;
            }
        }
        free(bd);
        free(bj);
    }
    return bad ? ORC_NO_MEM : ORC_OK;
}

/*
 * Per-row rho, sigma and directed weights (smooth kNN distances).
 * idx [n, k] int32, dist [n, k] double (ascending per row, as kNN returns).
 * Outputs rho[n], sigma[n], w[n, k]; iters[n] = bisection steps taken;
 * stop_margin[n] = min over steps of | |psum - target| - 1e-5 | (how close a
 * step came to flipping the stop test); floored[n] = 1 when the 1e-3 floor set
 * sigma; converged[n] = 1 when the stop test was met.
 */
int oracle_smooth_knn(const int32_t *idx, const double *dist, int64_t n, int k,
                      double *rho, double *sigma, double *w, int32_t *iters,
                      double *stop_margin, int32_t *floored, int32_t *converged) {
    if (!idx || !dist || n <= 0 || k <= 0) return ORC_BAD_ARG;
    const double target = log2((double)k);   /* bandwidth 1 */
    const double tol = 1e-5;
    const int n_iter = 64;
    const double floor_scale = 1e-3;

    double total = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) total += dist[(size_t)i * k + c];
    const double mean_all = total / ((double)n * (double)k);

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double *di = dist + (size_t)i * k;
        /* rho: first (smallest) non-zero distance of the row */
        double r = 0.0;
        for (int c = 0; c < k; ++c) {
            if (di[c] > 0.0) { r = di[c]; break; }
        }
        double lo = 0.0, hi = INFINITY, mid = 1.0, margin = INFINITY;
        int it = 0, conv = 0;
        for (it = 0; it < n_iter; ++it) {
            double psum = 0.0;
            for (int c = 1; c < k; ++c) {
                double g = di[c] - r;
                psum += (g > 0.0) ? exp(-(g / mid)) : 1.0;
            }
            double err = fabs(psum - target);
            double m = fabs(err - tol);
            if (m < margin) margin = m;
            if (err < tol) { conv = 1; ++it; break; }
            if (psum > target) {
                hi = mid;
                mid = (lo + hi) / 2.0;
            } else {
                lo = mid;
                mid = isinf(hi) ? mid * 2.0 : (lo + hi) / 2.0;
            }
        }
        double s = mid;
        int fl = 0;
        double row_mean = 0.0;
        for (int c = 0; c < k; ++c) row_mean += di[c];
        row_mean /= (double)k;
        double fl_val = (r > 0.0) ? floor_scale * row_mean : floor_scale * mean_all;
        if (s < fl_val) { s = fl_val; fl = 1; }
        rho[i] = r;
        sigma[i] = s;
        if (iters) iters[i] = it;
        if (stop_margin) stop_margin[i] = margin;
        if (floored) floored[i] = fl;
        if (converged) converged[i] = conv;
        for (int c = 0; c < k; ++c) {
            double v;
            if ((int64_t)idx[(size_t)i * k + c] == i) v = 0.0;
            else if (di[c] - r <= 0.0 || s == 0.0) v = 1.0;
            else v = exp(-((di[c] - r) / s));
            w[(size_t)i * k + c] = v;
        }
    }
    return ORC_OK;
}

/* weight of the directed edge i -> j, 0 when j is not in row i's list */
static double directed(const int32_t *idx, const double *w, int k, int64_t i, int64_t j) {
    for (int c = 0; c < k; ++c)
        if ((int64_t)idx[(size_t)i * k + c] == j) return w[(size_t)i * k + c];
    return 0.0;
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/*
 * Fuzzy union G = A + A^T - A o A^T of the directed weights (set-operation mix
 * ratio 1), as CSR with ascending columns, diagonal and zeros removed.
 * Rows of idx may hold -1 (no neighbour); such slots are ignored.
 * indptr [n+1] int64; indices/data of capacity `cap`; returns ORC_CAPACITY if
 * nnz exceeds cap (indptr still complete).
 */
int oracle_fuzzy_union(const int32_t *idx, const double *w, int64_t n, int k,
                       int64_t *indptr, int32_t *indices, double *data, int64_t cap) {
    if (!idx || !w || n <= 0 || k <= 0 || !indptr) return ORC_BAD_ARG;
    /* in-lists: for every j, the rows i that list j (built sequentially) */
    int64_t *in_cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!in_cnt) return ORC_NO_MEM;
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) {
            int64_t j = idx[(size_t)i * k + c];
            if (j >= 0 && j < n) in_cnt[j + 1]++;
        }
    for (int64_t j = 0; j < n; ++j) in_cnt[j + 1] += in_cnt[j];
    int64_t *in_src = (int64_t *)malloc(sizeof(int64_t) * (size_t)(in_cnt[n] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!in_src || !fill) { free(in_cnt); free(in_src); free(fill); return ORC_NO_MEM; }
    memcpy(fill, in_cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) {
            int64_t j = idx[(size_t)i * k + c];
            if (j >= 0 && j < n) in_src[fill[j]++] = i;
        }
    int64_t *cols = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1) * 1);
    int64_t cols_cap = k + 1;
    int status = ORC_OK;
    int64_t nnz = 0;
    indptr[0] = 0;
    for (int64_t i = 0; i < n && cols; ++i) {
        /* candidate columns: own list plus rows listing i */
        int64_t need = k + (in_cnt[i + 1] - in_cnt[i]);
        if (need > cols_cap) {
            int64_t *nc = (int64_t *)realloc(cols, sizeof(int64_t) * (size_t)need);
            if (!nc) { free(cols); cols = NULL; break; }
            cols = nc;
            cols_cap = need;
        }
        int64_t m = 0;
        for (int c = 0; c < k; ++c) {
            int64_t j = idx[(size_t)i * k + c];
            if (j >= 0 && j < n) cols[m++] = j;
        }
        for (int64_t p = in_cnt[i]; p < in_cnt[i + 1]; ++p) cols[m++] = in_src[p];
        qsort(cols, (size_t)m, sizeof(int64_t), cmp_i64);
        for (int64_t p = 0; p < m; ++p) {
            int64_t j = cols[p];
            if (p > 0 && cols[p - 1] == j) continue;   /* unique */
            if (j == i) continue;                      /* no diagonal */
            double a = directed(idx, w, k, i, j);
            double b = directed(idx, w, k, j, i);
            double g = a + b - a * b;
            if (g == 0.0) continue;                    /* no explicit zeros */
            if (nnz < cap && indices && data) {
                indices[nnz] = (int32_t)j;
                data[nnz] = g;
            } else {
                status = ORC_CAPACITY;
            }
            ++nnz;
        }
        indptr[i + 1] = nnz;
    }
    if (!cols) status = ORC_NO_MEM;
    free(cols);
    free(in_cnt);
    free(in_src);
    free(fill);
    return status;
}

/* ------------------------------------------------------------------------
 * Partitioner MLP (reference for the GPU training kernels).
 *
 * Layers: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3;
 * loss = mean over the batch of -sum_p t_p log softmax(z)_p (soft targets).
 * W1 [H1, D], W2 [H2, H1], W3 [P, H2] row-major (out x in).  With bf16 != 0
 * every GEMM operand that is a weight or an activation (x, h1, h2) is first
 * rounded to bfloat16 (round to nearest, ties to even), as the GPU does; the
 * arithmetic itself is double.  Gradients are of the loss with respect to
 * the (unrounded) parameters, treating the rounding as the identity
 * (straight-through), which is what the GPU backward computes.
 * ---------------------------------------------------------------------- */
static double round_bf16(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;   /* inf / nan unchanged */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

static double rd(double v, int bf16) { return bf16 ? round_bf16(v) : v; }

int oracle_mlp_loss_grad(const float *X, const float *T, int64_t B, int D, int H1, int H2, int P,
                         const float *params, int bf16, double *loss, double *grad) {
    if (!X || !T || !params || B <= 0 || D <= 0 || H1 <= 0 || H2 <= 0 || P <= 0) return ORC_BAD_ARG;
    const float *W1 = params, *b1 = W1 + (size_t)H1 * D;
    const float *W2 = b1 + H1, *b2 = W2 + (size_t)H2 * H1;
    const float *W3 = b2 + H2, *b3 = W3 + (size_t)P * H2;
    size_t np = (size_t)H1 * D + H1 + (size_t)H2 * H1 + H2 + (size_t)P * H2 + P;
    double *g = grad;
    if (g) memset(g, 0, sizeof(double) * np);
    double *gW1 = g, *gb1 = g ? g + (size_t)H1 * D : NULL;
    double *gW2 = g ? gb1 + H1 : NULL, *gb2 = g ? gW2 + (size_t)H2 * H1 : NULL;
    double *gW3 = g ? gb2 + H2 : NULL, *gb3 = g ? gW3 + (size_t)P * H2 : NULL;
    double *z1 = malloc(sizeof(double) * H1), *h1 = malloc(sizeof(double) * H1);
    double *z2 = malloc(sizeof(double) * H2), *h2 = malloc(sizeof(double) * H2);
    double *z3 = malloc(sizeof(double) * P), *dz3 = malloc(sizeof(double) * P);
    double *dh2 = malloc(sizeof(double) * H2), *dz2 = malloc(sizeof(double) * H2);
    double *dh1 = malloc(sizeof(double) * H1), *dz1 = malloc(sizeof(double) * H1);
    double *xr = malloc(sizeof(double) * D);
    if (!z1 || !h1 || !z2 || !h2 || !z3 || !dz3 || !dh2 || !dz2 || !dh1 || !dz1 || !xr) {
        free(z1); free(h1); free(z2); free(h2); free(z3); free(dz3); free(dh2); free(dz2); free(dh1); free(dz1); free(xr);
        return ORC_NO_MEM;
    }
    double total = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        const float *x = X + (size_t)b * D;
        const float *t = T + (size_t)b * P;
        for (int i = 0; i < D; ++i) xr[i] = rd(x[i], bf16);
        for (int o = 0; o < H1; ++o) {
            double s = 0.0;
            for (int i = 0; i < D; ++i) s += rd(W1[(size_t)o * D + i], bf16) * xr[i];
            z1[o] = s + b1[o];
            h1[o] = z1[o] > 0.0 ? z1[o] : 0.0;
        }
        for (int o = 0; o < H2; ++o) {
            double s = 0.0;
            for (int i = 0; i < H1; ++i) s += rd(W2[(size_t)o * H1 + i], bf16) * rd(h1[i], bf16);
            z2[o] = s + b2[o];
            h2[o] = z2[o] > 0.0 ? z2[o] : 0.0;
        }
        double zmax = -INFINITY;
        for (int o = 0; o < P; ++o) {
            double s = 0.0;
            for (int i = 0; i < H2; ++i) s += rd(W3[(size_t)o * H2 + i], bf16) * rd(h2[i], bf16);
            z3[o] = s + b3[o];
            if (z3[o] > zmax) zmax = z3[o];
        }
        double se = 0.0;
        for (int o = 0; o < P; ++o) se += exp(z3[o] - zmax);
        const double lse = zmax + log(se);
        double lb = 0.0;
        for (int o = 0; o < P; ++o) lb -= (double)t[o] * (z3[o] - lse);
        total += lb;
        if (!g) continue;
        double tsum = 0.0;
        for (int o = 0; o < P; ++o) tsum += (double)t[o];
        for (int o = 0; o < P; ++o) dz3[o] = (exp(z3[o] - lse) * tsum - (double)t[o]) / (double)B;
        for (int o = 0; o < P; ++o) {
            gb3[o] += dz3[o];
            for (int i = 0; i < H2; ++i) gW3[(size_t)o * H2 + i] += dz3[o] * rd(h2[i], bf16);
        }
        for (int i = 0; i < H2; ++i) {
            double s = 0.0;
            for (int o = 0; o < P; ++o) s += dz3[o] * rd(W3[(size_t)o * H2 + i], bf16);
            dh2[i] = s;
            dz2[i] = z2[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < H2; ++o) {
            gb2[o] += dz2[o];
            for (int i = 0; i < H1; ++i) gW2[(size_t)o * H1 + i] += dz2[o] * rd(h1[i], bf16);
        }
        for (int i = 0; i < H1; ++i) {
            double s = 0.0;
            for (int o = 0; o < H2; ++o) s += dz2[o] * rd(W2[(size_t)o * H1 + i], bf16);
            dh1[i] = s;
            dz1[i] = z1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < H1; ++o) {
            gb1[o] += dz1[o];
            for (int i = 0; i < D; ++i) gW1[(size_t)o * D + i] += dz1[o] * xr[i];
        }
    }
    *loss = total / (double)B;
    free(z1); free(h1); free(z2); free(h2); free(z3); free(dz3); free(dh2); free(dz2); free(dh1); free(dz1); free(xr);
    return ORC_OK;
}

/* ------------------------------------------------------------------ UMAP layout
 *
 * Edge-sampled stochastic gradient layout of the graph (the UMAP method of
 * McInnes, Healy & Melville 2018, section "Optimizing the embedding"; the
 * paper runs UMAP on the neighbourhood graph, Methods, "Dimensionality
 * reduction and graph analysis").  Low-dimensional similarity
 * phi(d) = 1 / (1 + a d^(2b)); every sampled graph entry pulls its head and
 * tail together along the gradient of log phi, and each sample draws
 * `neg_rate` vertices uniformly that push the head away along the gradient of
 * gamma log(1 - phi), the squared distance offset by 0.001.  Moves are
 * clipped to [-4, 4] per coordinate and scaled by the learning rate.
 *
 * Readings (the paper gives no layout algorithm of its own):
 *   - epochs n = 1 .. N with alpha_n = lr (1 - (n - 1) / N);
 *   - entry e of weight w_e is sampled in epoch n when
 *     floor(n f_e) > floor((n - 1) f_e), f_e = w_e / max w, so it is sampled
 *     floor(N f_e) times in N epochs (the epochs-per-sample schedule); f_e
 *     and the products n f_e are single precision, as the GPU takes them;
 *   - every sampled entry draws exactly neg_rate negative vertices; the q-th
 *     of entry e in epoch n is vertex h * n_vertices >> 32, h the high (q
 *     even) or low (q odd) 32 bits of output number
 *     ((n - 1) nnz + e) ceil(neg_rate / 2) + floor(q / 2) + 1 of SplitMix64
 *     seeded with `seed` (Steele, Lea & Flood 2014);
 *   - no move when the squared distance is 0 (the head itself, or a vertex
 *     at the same position);
 *   - an epoch reads the positions it started with: the moves of all its
 *     samples are summed and applied together at the end of the epoch.
 */
static uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (i >= 1) of SplitMix64 started from `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) {
    return splitmix64_mix(seed + i * 0x9E3779B97F4A7C15ULL);
}

/* Negative vertex q of entry e in epoch n (1-based), uniform on [0, nv):
 * negatives 2h and 2h + 1 use the high and the low 32 bits of one output. */
int64_t oracle_umap_negative(uint64_t seed, int epoch, int64_t nnz, int64_t e, int neg_rate, int q, int64_t nv) {
    const uint64_t pairs = (uint64_t)(neg_rate + 1) / 2;
    const uint64_t ctr = ((uint64_t)(epoch - 1) * (uint64_t)nnz + (uint64_t)e) * pairs + (uint64_t)(q / 2);
    const uint64_t u = oracle_splitmix64(seed, ctr + 1);
    const uint64_t half = (q % 2 == 0) ? (u >> 32) : (u & 0xFFFFFFFFULL);
    return (int64_t)((half * (uint64_t)nv) >> 32);
}

static double clip4(double v) { return v > 4.0 ? 4.0 : (v < -4.0 ? -4.0 : v); }

/* Entry e sampled in epoch n (single-precision schedule). */
static int umap_sampled(float w, float wmax, int epoch) {
    const float f = w / wmax;
    const float now = (float)epoch * f;
    const float before = (float)(epoch - 1) * f;
    return floorf(now) > floorf(before);
}

/*
 * Epochs first .. last (1-based, inclusive) of an N-epoch layout.
 * CSR graph (indptr [n+1], indices, data [nnz], weights > 0 expected);
 * Y [n, dim] double, updated in place.  absmove [n] (nullable) receives, for
 * the last epoch run, the sum of |move| over every coordinate of every move
 * applied to the vertex (for tolerances); samples [nnz] (nullable, int64) is
 * incremented once per epoch in which the entry was sampled.  mask [n]
 * (nullable) restricts one epoch to the masked vertices: only they move, and
 * only moves onto them are computed (first must equal last).
 */
int oracle_umap_epochs(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n, int dim,
                       double *Y, double a, double b, double gamma, double lr, int neg_rate, int n_epochs,
                       int first, int last, uint64_t seed, const uint8_t *mask, double *absmove,
                       int64_t *samples) {
    if (!indptr || !Y || n <= 0 || dim < 1 || dim > 16 || neg_rate < 0 || n_epochs < 1 || first < 1 ||
        last > n_epochs || (mask && first != last))
        return ORC_BAD_ARG;
    const int64_t nnz = indptr[n];
    if (nnz > 0 && (!indices || !data)) return ORC_BAD_ARG;
    float wmax = 0.f;
    for (int64_t e = 0; e < nnz; ++e)
        if (data[e] > wmax) wmax = data[e];
    double *delta = (double *)calloc((size_t)n * dim, sizeof(double));
    double *am = (double *)calloc((size_t)n, sizeof(double));
    if (!delta || !am) { free(delta); free(am); return ORC_NO_MEM; }
    for (int epoch = first; epoch <= last; ++epoch) {
        const double alpha = lr * (1.0 - (double)(epoch - 1) / (double)n_epochs);
        memset(delta, 0, sizeof(double) * (size_t)n * dim);
        memset(am, 0, sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) {
                if (!(wmax > 0.f) || !umap_sampled(data[e], wmax, epoch)) continue;
                if (samples) samples[e]++;
                const int64_t j = indices[e];
                const int head = !mask || mask[i], tail = !mask || mask[j];
                const double *yi = Y + (size_t)i * dim;
                if (head || tail) {   /* attraction: head and tail move */
                    const double *yj = Y + (size_t)j * dim;
                    double d2 = 0.0;
                    for (int t = 0; t < dim; ++t) d2 += (yi[t] - yj[t]) * (yi[t] - yj[t]);
                    if (d2 > 0.0) {
                        const double c = -2.0 * a * b * pow(d2, b - 1.0) / (1.0 + a * pow(d2, b));
                        for (int t = 0; t < dim; ++t) {
                            const double m = alpha * clip4(c * (yi[t] - yj[t]));
                            if (head) { delta[(size_t)i * dim + t] += m; am[i] += fabs(m); }
                            if (tail) { delta[(size_t)j * dim + t] -= m; am[j] += fabs(m); }
                        }
                    }
                }
                if (!head) continue;
                for (int q = 0; q < neg_rate; ++q) {   /* repulsion: only the head moves */
                    const int64_t v = oracle_umap_negative(seed, epoch, nnz, e, neg_rate, q, n);
                    const double *yv = Y + (size_t)v * dim;
                    double d2 = 0.0;
                    for (int t = 0; t < dim; ++t) d2 += (yi[t] - yv[t]) * (yi[t] - yv[t]);
                    if (!(d2 > 0.0)) continue;
                    const double c = 2.0 * gamma * b / ((0.001 + d2) * (1.0 + a * pow(d2, b)));
                    for (int t = 0; t < dim; ++t) {
                        const double m = alpha * clip4(c * (yi[t] - yv[t]));
                        delta[(size_t)i * dim + t] += m;
                        am[i] += fabs(m);
                    }
                }
            }
        }
        for (int64_t v = 0; v < n; ++v)
            if (!mask || mask[v])
                for (int t = 0; t < dim; ++t) Y[(size_t)v * dim + t] += delta[(size_t)v * dim + t];
    }
    if (absmove) memcpy(absmove, am, sizeof(double) * (size_t)n);
    free(delta);
    free(am);
    return ORC_OK;
}

/* ------------------------------------------------------------------ E-distance
 *
 * Energy distance between groups of cells (paper, Methods, "Perturbation
 * distance computation"): E(X, Y) = 2 mean ||X_i - Y_j|| - mean ||X_i - X_i'||
 * - mean ||Y_j - Y_j'||, Euclidean distances over the embedding.  Groups are
 * CSR-style: group g holds the cells cell_index[offsets[g] .. offsets[g+1])
 * (cell_index NULL: the rows themselves).  For a pair a != b the sum runs over
 * every i in a and j in b; for a == b over the pairs i < j of positions in the
 * group (the upper triangle), as the paper's kernel accumulates them.
 */
static double row_dist(const float *X, int d, int64_t a, int64_t b) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        const double v = (double)X[(size_t)a * d + t] - (double)X[(size_t)b * d + t];
        s += v * v;
    }
    return sqrt(s);
}

/* Distance sums of the requested pairs (pairs [n_pairs][2], a <= b; NULL: all
 * pairs a <= b), written to sums[a * G + b] (other entries untouched). */
int oracle_edistance_sums(const float *X, int64_t n_rows, int d, const int32_t *cell_index, const int64_t *offsets,
                          int G, const int32_t *pairs, int64_t n_pairs, double *sums) {
    if (!X || n_rows <= 0 || d <= 0 || !offsets || G <= 0 || !sums) return ORC_BAD_ARG;
    const int64_t np = pairs ? n_pairs : (int64_t)G * (G + 1) / 2;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p) {
        int a, b;
        if (pairs) {
            a = pairs[2 * p];
            b = pairs[2 * p + 1];
        } else {   /* p-th pair of the upper triangle, row by row */
            int64_t r = p;
            a = 0;
            while (r >= G - a) { r -= G - a; ++a; }
            b = a + (int)r;
        }
        if (a < 0 || b >= G || a > b) { bad = 1; continue; }
        double s = 0.0;
        for (int64_t u = offsets[a]; u < offsets[a + 1]; ++u) {
            const int64_t i = cell_index ? cell_index[u] : u;
            const int64_t v0 = (a == b) ? u + 1 : offsets[b];
            for (int64_t v = v0; v < offsets[b + 1]; ++v) {
                const int64_t j = cell_index ? cell_index[v] : v;
                s += row_dist(X, d, i, j);
            }
        }
        sums[(size_t)a * G + b] = s;
    }
    return bad ? ORC_BAD_ARG : ORC_OK;
}

/* Mean distances and energy distances from the sums of every pair a <= b:
 * mean[a][b] = sums / (n_a n_b) (a != b) or sums / (n_a (n_a - 1) / 2)
 * (a == b; 0 for a group of fewer than two cells, whose diagonal the paper's
 * kernel skips); E[a][b] = E[b][a] = 2 mean[a][b] - mean[a][a] - mean[b][b]. */
int oracle_edistance_assemble(const int64_t *offsets, int G, const double *sums, double *mean, double *E) {
    if (!offsets || G <= 0 || !sums || !mean || !E) return ORC_BAD_ARG;
    for (int a = 0; a < G; ++a)
        for (int b = a; b < G; ++b) {
            const double na = (double)(offsets[a + 1] - offsets[a]), nb = (double)(offsets[b + 1] - offsets[b]);
            double m;
            if (a == b) m = na >= 2 ? sums[(size_t)a * G + a] / (na * (na - 1.0) / 2.0) : 0.0;
            else m = (na > 0 && nb > 0) ? sums[(size_t)a * G + b] / (na * nb) : 0.0;
            mean[(size_t)a * G + b] = mean[(size_t)b * G + a] = m;
        }
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b)
            E[(size_t)a * G + b] = 2.0 * mean[(size_t)a * G + b] - mean[(size_t)a * G + a] - mean[(size_t)b * G + b];
    return ORC_OK;
}

/*
 * Approximate kNN by NN-descent (Dong, Charikar & Li, "Efficient k-nearest
 * neighbor graph construction for generic similarity measures", WWW 2011):
 * a neighbour of a neighbour is probably a neighbour, so every list is
 * improved by joining, around each point v, the points v's list and reverse
 * list name.  This is the synchronous form with deterministic sampling that
 * the library runs (the paper names PyNNDescent as its CPU neighbour search,
 * Methods, "Benchmarking", and prints no algorithm); every step below is a
 * reading of the method and is the definition both sides follow.
 *
 *   delta2(a, b): FP32 squared Euclidean distance, acc = 0, then for
 *     t = 0 .. d-1: u = x_a[t] - x_b[t] (FP32), acc = fmaf(u, u, acc).
 *     (Symmetric bit for bit: x_b - x_a = -(x_a - x_b) exactly.)
 *   key(x, id) = (bits of x) << 32 | id: lists are ordered by (delta2, id);
 *     a non-negative float's bits order like its value.
 *   G(i) = output i (i >= 1) of SplitMix64 seeded with `seed`.
 *   slot_b(id) = (uint32)(id * 0x9E3779B1) >> (32 - b) (Fibonacci hashing;
 *     0 when b = 0, a single slot).
 *
 * Initial lists: u itself, then (with caller lists init [n, k]) the entries
 * of init[u] in order that lie in [0, n) and are not yet present, then the
 * distinct values of (u + 1 + G(u 2k + j + 1) mod (n - 1)) mod n for
 * j = 0 .. 2k - 1, then u + 1, u + 2, ... mod n not yet present, each step
 * only while the list is short of k; ordered by key.  Every entry but u is
 * flagged new.
 *
 * Iteration t (0-based), all steps reading the lists B_t as they were when
 * the iteration began:
 *   1. Forward samples.  new_f(u): the first S entries (list order) flagged
 *      new, u itself excluded; their flags are cleared.  old_f(u): the
 *      entries flagged old before that, u excluded.
 *   2. Reverse samples.  R (power of two) slots per point for new and for
 *      old: source u offers the key p(t, u) << 32 | u, p(t, u) the high 32
 *      bits of G(((t + 1) << 40) | u), to slot slot_logR(u) of every w in
 *      new_f(u) (resp. old_f(u)); a slot keeps its smallest key.  The ids in
 *      w's new (resp. old) slots are w's reverse samples.
 *   3. Join lists.  new(v) = new_f(v) united with v's new reverse samples;
 *      old(v) = (old_f(v) united with v's old reverse samples) minus new(v).
 *   4. Local join.  For every v and every unordered pair {a, b}, a != b,
 *      with a in new(v) and b in new(v) or old(v): x = delta2(a, b); if
 *      key(x, b) < thr(a) (the key of the last entry of B_t(a)) then
 *      C(a)[slot_logC(b)] = min(C(a)[...], key(x, b)); the same for b with a.
 *      (A candidate at or above thr(a) could never enter a's list, so the
 *      test only spares slots.)  C slots per point start empty.
 *   5. Merge.  B_{t+1}(u) = the k smallest distinct keys of B_t(u) and u's
 *      non-empty candidate slots (equal keys are one entry: same id, same
 *      distance); entries that were in B_t keep their flag, the others are
 *      flagged new.  changes_t = number of entries not in B_t, summed over u.
 *   6. Stop after iteration t when changes_t < delta n k.
 * Output: ids in key order and dist = sqrtf(delta2).
 */
static float nd_delta2(const float *X, int d, int64_t a, int64_t b) {
    float acc = 0.0f;
    for (int t = 0; t < d; ++t) {
        const float u = X[(size_t)a * d + t] - X[(size_t)b * d + t];
        acc = fmaf(u, u, acc);
    }
    return acc;
}

static uint64_t nd_key(float x, int64_t id) {
    uint32_t bits;
    memcpy(&bits, &x, sizeof bits);
    return ((uint64_t)bits << 32) | (uint32_t)id;
}

static uint32_t nd_slot(int64_t id, int bits) {
    return bits == 0 ? 0u : (uint32_t)((uint32_t)id * 0x9E3779B1u) >> (32 - bits);
}

static int nd_log2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return (1 << b) == v ? b : -1;
}

static int cmp_u64(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* One pool entry of the merge: key, then 0 for a list entry / 1 for a
 * candidate (so a list entry comes first among equal keys), and its flag. */
typedef struct {
    uint64_t key;
    int src;
    int isnew;
} nd_item;

static int cmp_item(const void *a, const void *b) {
    const nd_item *x = (const nd_item *)a, *y = (const nd_item *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->src - y->src;
}

static int nd_has(const int64_t *v, int m, int64_t x) {
    for (int i = 0; i < m; ++i)
        if (v[i] == x) return 1;
    return 0;
}

/*
 * X [n, d] float32; init [n, k] int32 caller lists or NULL; k list length
 * (self included), 2 <= k <= n; S new samples
 * per list (1 <= S <= k); R reverse slots and C candidate slots (powers of
 * two); T iterations at most; delta >= 0.  Outputs idx [n, k], d2 [n, k]
 * (the FP32 squared distances), changes [T] (0 for iterations not run),
 * pairs [T] (pairs joined per iteration; nullable) and iters_run (nullable).
 */
int oracle_nndescent(const float *X, int64_t n, int d, int k, int S, int R, int C, int T, double delta,
                     uint64_t seed, const int32_t *init, int32_t *idx, float *d2, int64_t *changes,
                     int64_t *pairs, int *iters_run) {
    const int lr = nd_log2(R), lc = nd_log2(C);
    if (!X || !idx || !d2 || n < 1 || d < 1 || k < 2 || k > n || S < 1 || S > k || lr < 0 || lc < 0 ||
        T < 0 || delta < 0)
        return ORC_BAD_ARG;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * k);
    unsigned char *isnew = (unsigned char *)malloc((size_t)n * k);
    int64_t *newf = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * S);
    int *nnew = (int *)malloc(sizeof(int) * (size_t)n);
    int64_t *oldf = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * k);
    int *nold = (int *)malloc(sizeof(int) * (size_t)n);
    uint64_t *rn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * R);
    uint64_t *ro = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * R);
    uint64_t *cand = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * C);
    uint64_t *thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int64_t *jn = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + R));
    int64_t *jo = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + R));
    nd_item *pool = (nd_item *)malloc(sizeof(nd_item) * (size_t)(k + C));
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!key || !isnew || !newf || !nnew || !oldf || !nold || !rn || !ro || !cand || !thr || !jn || !jo || !pool ||
        !ids) {
        free(key); free(isnew); free(newf); free(nnew); free(oldf); free(nold); free(rn); free(ro);
        free(cand); free(thr); free(jn); free(jo); free(pool); free(ids);
        return ORC_NO_MEM;
    }
    /* initial lists */
    for (int64_t u = 0; u < n; ++u) {
        int m = 0;
        ids[m++] = u;
        if (init)
            for (int c = 0; c < k && m < k; ++c) {
                const int64_t r = init[(size_t)u * k + c];
                if (r >= 0 && r < n && !nd_has(ids, m, r)) ids[m++] = r;
            }
        for (int j = 0; j < 2 * k && m < k; ++j) {
            const uint64_t g = oracle_splitmix64(seed, (uint64_t)u * (uint64_t)(2 * k) + (uint64_t)j + 1);
            const int64_t r = (u + 1 + (int64_t)(g % (uint64_t)(n - 1))) % n;
            if (!nd_has(ids, m, r)) ids[m++] = r;
        }
        for (int64_t s = 1; m < k; ++s) {
            const int64_t r = (u + s) % n;
            if (!nd_has(ids, m, r)) ids[m++] = r;
        }
        for (int c = 0; c < k; ++c) key[(size_t)u * k + c] = nd_key(nd_delta2(X, d, u, ids[c]), ids[c]);
        qsort(key + (size_t)u * k, (size_t)k, sizeof(uint64_t), cmp_u64);
        for (int c = 0; c < k; ++c)
            isnew[(size_t)u * k + c] = (int64_t)(uint32_t)key[(size_t)u * k + c] != u;
    }
    if (changes)
        for (int t = 0; t < T; ++t) changes[t] = 0;
    if (pairs)
        for (int t = 0; t < T; ++t) pairs[t] = 0;
    int run = 0;
    for (int t = 0; t < T; ++t) {
        /* 1. forward samples */
        for (int64_t u = 0; u < n; ++u) {
            int a = 0, o = 0;
            for (int c = 0; c < k; ++c) {
                const size_t e = (size_t)u * k + c;
                const int64_t id = (int64_t)(uint32_t)key[e];
                if (id == u) continue;
                if (isnew[e]) {
                    if (a < S) {
                        newf[(size_t)u * S + a++] = id;
                        isnew[e] = 0;
                    }
                } else {
                    oldf[(size_t)u * k + o++] = id;
                }
            }
            nnew[u] = a;
            nold[u] = o;
        }
        /* 2. reverse samples */
        for (size_t e = 0; e < (size_t)n * R; ++e) rn[e] = ro[e] = UINT64_MAX;
        for (int64_t u = 0; u < n; ++u) {
            const uint64_t p = oracle_splitmix64(seed, ((uint64_t)(t + 1) << 40) | (uint64_t)u) >> 32;
            const uint64_t pk = (p << 32) | (uint32_t)u;
            const uint32_t s = nd_slot(u, lr);
            for (int i = 0; i < nnew[u]; ++i) {
                uint64_t *q = rn + (size_t)newf[(size_t)u * S + i] * R + s;
                if (pk < *q) *q = pk;
            }
            for (int i = 0; i < nold[u]; ++i) {
                uint64_t *q = ro + (size_t)oldf[(size_t)u * k + i] * R + s;
                if (pk < *q) *q = pk;
            }
        }
        /* 3-4. join lists and local join */
        for (size_t e = 0; e < (size_t)n * C; ++e) cand[e] = UINT64_MAX;
        for (int64_t u = 0; u < n; ++u) thr[u] = key[(size_t)u * k + k - 1];
        for (int64_t v = 0; v < n; ++v) {
            int a = 0, o = 0;
            for (int i = 0; i < nnew[v]; ++i)
                if (!nd_has(jn, a, newf[(size_t)v * S + i])) jn[a++] = newf[(size_t)v * S + i];
            for (int s = 0; s < R; ++s) {
                const uint64_t q = rn[(size_t)v * R + s];
                if (q != UINT64_MAX && !nd_has(jn, a, (int64_t)(uint32_t)q)) jn[a++] = (int64_t)(uint32_t)q;
            }
            for (int i = 0; i < nold[v]; ++i) {
                const int64_t id = oldf[(size_t)v * k + i];
                if (!nd_has(jn, a, id) && !nd_has(jo, o, id)) jo[o++] = id;
            }
            for (int s = 0; s < R; ++s) {
                const uint64_t q = ro[(size_t)v * R + s];
                if (q == UINT64_MAX) continue;
                const int64_t id = (int64_t)(uint32_t)q;
                if (!nd_has(jn, a, id) && !nd_has(jo, o, id)) jo[o++] = id;
            }
            if (pairs) pairs[t] += (int64_t)a * (a - 1) / 2 + (int64_t)a * o;
            for (int i = 0; i < a; ++i)
                for (int j = i + 1; j < a + o; ++j) {
                    const int64_t pa = jn[i], pb = (j < a) ? jn[j] : jo[j - a];
                    const float x = nd_delta2(X, d, pa, pb);
                    const uint64_t ka = nd_key(x, pb), kb = nd_key(x, pa);
                    if (ka < thr[pa]) {
                        uint64_t *q = cand + (size_t)pa * C + nd_slot(pb, lc);
                        if (ka < *q) *q = ka;
                    }
                    if (kb < thr[pb]) {
                        uint64_t *q = cand + (size_t)pb * C + nd_slot(pa, lc);
                        if (kb < *q) *q = kb;
                    }
                }
        }
        /* 5. merge */
        int64_t ch = 0;
        for (int64_t u = 0; u < n; ++u) {
            int m = 0;
            for (int c = 0; c < k; ++c) {
                pool[m].key = key[(size_t)u * k + c];
                pool[m].src = 0;
                pool[m++].isnew = isnew[(size_t)u * k + c];
            }
            for (int s = 0; s < C; ++s) {
                const uint64_t q = cand[(size_t)u * C + s];
                if (q == UINT64_MAX) continue;
                pool[m].key = q;
                pool[m].src = 1;
                pool[m++].isnew = 1;
            }
            qsort(pool, (size_t)m, sizeof(nd_item), cmp_item);
            int w = 0;
            for (int i = 0; i < m && w < k; ++i) {
                if (i > 0 && pool[i].key == pool[i - 1].key) continue;
                key[(size_t)u * k + w] = pool[i].key;
                isnew[(size_t)u * k + w] = (unsigned char)pool[i].isnew;
                ch += pool[i].src;
                ++w;
            }
        }
        if (changes) changes[t] = ch;
        ++run;
        if ((double)ch < delta * (double)n * (double)k) break;
    }
    for (size_t e = 0; e < (size_t)n * k; ++e) {
        idx[e] = (int32_t)(uint32_t)key[e];
        const uint32_t bits = (uint32_t)(key[e] >> 32);
        memcpy(&d2[e], &bits, sizeof bits);
    }
    if (iters_run) *iters_run = run;
    free(key); free(isnew); free(newf); free(nnew); free(oldf); free(nold); free(rn); free(ro);
    free(cand); free(thr); free(jn); free(jo); free(pool); free(ids);
    return ORC_OK;
}

/*
 * Leiden community detection (Traag, Waltman & van Eck, "From Louvain to
 * Leiden: guaranteeing well-connected communities", Sci. Rep. 2019), the
 * clustering the paper runs on the stored graph (Methods, "Dimensionality
 * reduction and graph analysis"), with the modularity quality function and a
 * resolution gamma, as scanpy calls it.  The library runs it synchronously
 * (every vertex decides on the state of the round before), so this is the
 * same synchronous form; the readings (beside the paper's steps) are:
 *
 *   Weights in fixed point: W = rint(w * 2^32) as a 64-bit integer, so every
 *   sum is exact and independent of its order; gamma enters as
 *   G = rint(gamma * 2^16).  Strength k_v = sum of v's row (a self-loop entry
 *   counted as stored), 2m = sum of all strengths, tot_c = sum of k over c.
 *   Moving v from community a to c changes the quality by a positive
 *   multiple of
 *     g(c) = s_c 2m 2^16 - G k_v tot_c        (c != a),
 *     g(a) = s_a 2m 2^16 - G k_v (tot_a - k_v) (staying),
 *   s_c = weight of v's entries to other vertices of c; compared exactly
 *   in 128-bit integers.  Entries whose fixed-point weight is 0 are skipped,
 *   so a vertex's candidate communities are those with s_c > 0.
 *   Labels are vertex ids; after each phase a community takes the smallest
 *   id among its members.
 *
 * 1. Local moving (the paper's MoveNodesFast), in rounds r = 0, 1, ...: each
 *    vertex picks the neighbouring community c != a with the largest g(c)
 *    (ties: smallest c) and moves there if g(c) > g(a) and, in even rounds,
 *    c < a, in odd rounds c > a (so two vertices never swap forever).  All
 *    moves of a round apply together.  The phase ends after two rounds in a
 *    row without a move, or after max_rounds rounds (8 by default).
 * 2. Refinement (RefinePartition / MergeNodesSubset): inside each community
 *    C of step 1, every vertex starts alone.  A vertex v that is still alone
 *    and well connected to C (s_{C-v} 2m 2^16 >= G k_v (tot_C - k_v)) looks at
 *    the subcommunities S of its neighbours in C that are well connected
 *    (ext_S 2m 2^16 >= G tot_S (tot_C - tot_S), ext_S the weight from S to
 *    C - S) and picks the one with the largest g(S) = s_S 2m 2^16 -
 *    G k_v tot_S >= 0 (ties: smallest label); the paper draws it at random
 *    with probability growing with the gain, and the greedy choice is its
 *    limit of zero randomness.  A vertex some other vertex picked stays (so
 *    merges never chain within a round); all other picks apply together;
 *    rounds repeat until none moves or max_rounds.
 * 3. Aggregation (AggregateGraph): one node per refined subcommunity, in the
 *    order of their smallest member; the weight between two nodes is the sum
 *    of the weights between their members (a node's self-loop holds its
 *    internal weight, both directions).  Each node starts in the community of
 *    step 1 that holds its members.
 * Levels repeat until step 1 leaves every community a single node, or the
 * refinement merges nothing, or max_levels.  n_iter such runs are made, each
 * starting from the previous partition (scanpy runs two).  Output: each
 * vertex's community, numbered by first appearance over the vertices.
 */
typedef __int128 ld_i128;

typedef struct {
    int64_t nv;
    int64_t *ip;
    int32_t *col;
    int64_t *wt;
} ld_graph;

static void ld_free(ld_graph *g) {
    free(g->ip);
    free(g->col);
    free(g->wt);
    g->ip = NULL;
    g->col = NULL;
    g->wt = NULL;
}

/* Relabels every community by its smallest member. */
static void ld_canon(int64_t nv, int32_t *lab, int32_t *tmp) {
    for (int64_t v = 0; v < nv; ++v) tmp[v] = INT32_MAX;
    for (int64_t v = 0; v < nv; ++v)
        if (v < tmp[lab[v]]) tmp[lab[v]] = (int32_t)v;
    for (int64_t v = 0; v < nv; ++v) lab[v] = tmp[lab[v]];
}

/* Step 1.  Returns the number of moves made; comm is relabelled. */
static int64_t ld_move(const ld_graph *g, const int64_t *k, int64_t m2, int64_t G, int max_rounds, int32_t *comm,
                       int64_t *tot, int64_t *s, int32_t *touched, int32_t *next) {
    const int64_t nv = g->nv;
    int64_t total = 0;
    int quiet = 0;
    for (int r = 0; r < max_rounds && quiet < 2; ++r) {
        for (int64_t c = 0; c < nv; ++c) tot[c] = 0;
        for (int64_t v = 0; v < nv; ++v) tot[comm[v]] += k[v];
        int64_t moves = 0;
        for (int64_t v = 0; v < nv; ++v) {
            const int32_t a = comm[v];
            int nt = 0;
            for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
                const int32_t u = g->col[e];
                if (u == v || g->wt[e] == 0) continue;
                const int32_t c = comm[u];
                if (s[c] == 0) touched[nt++] = c;
                s[c] += g->wt[e];
            }
            const ld_i128 ga = (ld_i128)s[a] * m2 * 65536 - (ld_i128)G * k[v] * (tot[a] - k[v]);
            int32_t best = -1;
            ld_i128 gb = 0;
            for (int i = 0; i < nt; ++i) {
                const int32_t c = touched[i];
                if (c == a) continue;
                const ld_i128 gc = (ld_i128)s[c] * m2 * 65536 - (ld_i128)G * k[v] * tot[c];
                if (best < 0 || gc > gb || (gc == gb && c < best)) {
                    best = c;
                    gb = gc;
                }
            }
            for (int i = 0; i < nt; ++i) s[touched[i]] = 0;
            next[v] = a;
            if (best >= 0 && gb > ga && ((r % 2 == 0) ? best < a : best > a)) {
                next[v] = best;
                ++moves;
            }
        }
        memcpy(comm, next, sizeof(int32_t) * (size_t)nv);
        total += moves;
        quiet = moves ? 0 : quiet + 1;
    }
    ld_canon(nv, comm, next);
    for (int64_t c = 0; c < nv; ++c) tot[c] = 0;
    for (int64_t v = 0; v < nv; ++v) tot[comm[v]] += k[v];
    return total;
}

/* Step 2: ref (labels = vertex ids) refined inside comm; relabelled. */
static void ld_refine(const ld_graph *g, const int64_t *k, int64_t m2, int64_t G, int max_rounds,
                      const int32_t *comm, const int64_t *tot, int32_t *ref, int64_t *s, int32_t *touched,
                      int32_t *target, int64_t *wC, int64_t *rtot, int64_t *ext, int32_t *size,
                      unsigned char *picked, int32_t *tmp) {
    const int64_t nv = g->nv;
    for (int64_t v = 0; v < nv; ++v) {
        ref[v] = (int32_t)v;
        int64_t w = 0;
        for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
            const int32_t u = g->col[e];
            if (u != v && comm[u] == comm[v]) w += g->wt[e];
        }
        wC[v] = w;
    }
    for (int r = 0; r < max_rounds; ++r) {
        /* subcommunity totals, sizes, external weights at the round start */
        for (int64_t S = 0; S < nv; ++S) {
            rtot[S] = 0;
            ext[S] = 0;
            size[S] = 0;
            picked[S] = 0;
        }
        for (int64_t v = 0; v < nv; ++v) {
            rtot[ref[v]] += k[v];
            size[ref[v]] += 1;
            int64_t wS = 0;
            for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
                const int32_t u = g->col[e];
                if (u != v && ref[u] == ref[v]) wS += g->wt[e];
            }
            ext[ref[v]] += wC[v] - wS;
        }
        for (int64_t v = 0; v < nv; ++v) {
            target[v] = -1;
            if (size[ref[v]] != 1) continue;   /* only vertices still alone move */
            const int32_t C = comm[v];
            if ((ld_i128)wC[v] * m2 * 65536 < (ld_i128)G * k[v] * (tot[C] - k[v])) continue;
            int nt = 0;
            for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
                const int32_t u = g->col[e];
                if (u == v || comm[u] != C || g->wt[e] == 0) continue;
                const int32_t S = ref[u];
                if (s[S] == 0) touched[nt++] = S;
                s[S] += g->wt[e];
            }
            int32_t best = -1;
            ld_i128 gb = 0;
            for (int i = 0; i < nt; ++i) {
                const int32_t S = touched[i];
                if (S == ref[v]) continue;
                if ((ld_i128)ext[S] * m2 * 65536 < (ld_i128)G * rtot[S] * (tot[C] - rtot[S])) continue;
                const ld_i128 gS = (ld_i128)s[S] * m2 * 65536 - (ld_i128)G * k[v] * rtot[S];
                if (gS < 0) continue;
                if (best < 0 || gS > gb || (gS == gb && S < best)) {
                    best = S;
                    gb = gS;
                }
            }
            for (int i = 0; i < nt; ++i) s[touched[i]] = 0;
            target[v] = best;
        }
        for (int64_t v = 0; v < nv; ++v)
            if (target[v] >= 0) picked[target[v]] = 1;
        int64_t moves = 0;
        for (int64_t v = 0; v < nv; ++v)
            if (target[v] >= 0 && !picked[ref[v]]) {
                ref[v] = target[v];
                ++moves;
            }
        if (!moves) break;
    }
    ld_canon(nv, ref, tmp);
}

/* Step 3: the graph of the refined subcommunities.  node[v] (out) = new index
 * of v's subcommunity; returns the node count (0 on allocation failure). */
static int64_t ld_aggregate(const ld_graph *g, const int32_t *ref, int32_t *node, ld_graph *out, int64_t *acc,
                            int32_t *touched) {
    const int64_t nv = g->nv;
    int64_t K = 0;
    for (int64_t v = 0; v < nv; ++v)
        if (ref[v] == v) node[v] = (int32_t)K++;   /* labels are smallest members: ascending order */
    for (int64_t v = 0; v < nv; ++v) node[v] = node[ref[v]];
    /* members of each node, in vertex order */
    int64_t *moff = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    out->ip = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    if (!moff || !mem || !out->ip) {
        free(moff);
        free(mem);
        return 0;
    }
    for (int64_t v = 0; v < nv; ++v) moff[node[v] + 1]++;
    for (int64_t c = 0; c < K; ++c) moff[c + 1] += moff[c];
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
        if (!cur) {
            free(moff);
            free(mem);
            return 0;
        }
        for (int64_t c = 0; c < K; ++c) cur[c] = moff[c];
        for (int64_t v = 0; v < nv; ++v) mem[cur[node[v]]++] = (int32_t)v;
        free(cur);
    }
    /* two passes: row lengths, then the rows (columns ascending) */
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t c = 0; c < K; ++c) {
            int nt = 0;
            for (int64_t i = moff[c]; i < moff[c + 1]; ++i) {
                const int32_t v = mem[i];
                for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
                    if (g->wt[e] == 0) continue;
                    const int32_t t = node[g->col[e]];
                    if (acc[t] == 0) touched[nt++] = t;
                    acc[t] += g->wt[e];
                }
            }
            /* ascending columns: insertion sort of the touched list */
            for (int i = 1; i < nt; ++i) {
                const int32_t x = touched[i];
                int j = i - 1;
                while (j >= 0 && touched[j] > x) {
                    touched[j + 1] = touched[j];
                    --j;
                }
                touched[j + 1] = x;
            }
            if (pass == 0) {
                out->ip[c + 1] = out->ip[c] + nt;
            } else {
                int64_t p = out->ip[c];
                for (int i = 0; i < nt; ++i) {
                    out->col[p] = touched[i];
                    out->wt[p++] = acc[touched[i]];
                }
            }
            for (int i = 0; i < nt; ++i) acc[touched[i]] = 0;
        }
        if (pass == 0) {
            out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(out->ip[K] > 0 ? out->ip[K] : 1));
            out->wt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(out->ip[K] > 0 ? out->ip[K] : 1));
            if (!out->col || !out->wt) {
                free(moff);
                free(mem);
                return 0;
            }
        }
    }
    out->nv = K;
    free(moff);
    free(mem);
    return K;
}

/*
 * Symmetric CSR graph (indptr [n + 1], indices, data [nnz], data > 0
 * expected; a zero weight adds nothing), resolution gamma, n_iter runs,
 * max_levels, max_rounds.  init [n] (nullable): starting partition labels in
 * [0, n).  Outputs membership [n] (communities numbered by first appearance),
 * *n_comm, *quality = sum_c (in_c / 2m - gamma (tot_c / 2m)^2) on the
 * fixed-point weights (nullable), *levels_run (levels of the last run).
 */
int oracle_leiden(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n, double gamma,
                  int n_iter, int max_levels, int max_rounds, const int32_t *init, int32_t *membership,
                  int64_t *n_comm, double *quality, int *levels_run) {
    if (!indptr || !membership || n < 1 || n >= INT32_MAX || gamma <= 0 || gamma >= 32768 || n_iter < 1 ||
        max_levels < 1 || max_rounds < 1)
        return ORC_BAD_ARG;
    const int64_t nnz = indptr[n];
    for (int64_t v = 0; v < n; ++v)
        if (indptr[v + 1] < indptr[v]) return ORC_BAD_ARG;
    for (int64_t e = 0; e < nnz; ++e)
        if (indices[e] < 0 || indices[e] >= n) return ORC_BAD_ARG;
    const int64_t G = (int64_t)llrint(gamma * 65536.0);
    ld_graph g0;
    g0.nv = n;
    g0.ip = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g0.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    g0.wt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    const size_t N = (size_t)n;
    int64_t *k = (int64_t *)malloc(sizeof(int64_t) * N), *tot = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *s = (int64_t *)calloc(N, sizeof(int64_t)), *wC = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *rtot = (int64_t *)malloc(sizeof(int64_t) * N), *ext = (int64_t *)malloc(sizeof(int64_t) * N);
    int32_t *comm = (int32_t *)malloc(sizeof(int32_t) * N), *next = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * N), *ref = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *target = (int32_t *)malloc(sizeof(int32_t) * N), *size = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *node = (int32_t *)malloc(sizeof(int32_t) * N), *top = (int32_t *)malloc(sizeof(int32_t) * N);
    unsigned char *picked = (unsigned char *)malloc(N);
    int rc = ORC_OK;
    if (!g0.ip || !g0.col || !g0.wt || !k || !tot || !s || !wC || !rtot || !ext || !comm || !next || !touched ||
        !ref || !target || !size || !node || !top || !picked) {
        rc = ORC_NO_MEM;
        goto done;
    }
    memcpy(g0.ip, indptr, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < nnz; ++e) {
        g0.col[e] = indices[e];
        g0.wt[e] = (int64_t)llrint((double)data[e] * 4294967296.0);
    }
    for (int64_t v = 0; v < n; ++v) membership[v] = init ? init[v] : (int32_t)v;
    for (int64_t v = 0; v < n; ++v)
        if (membership[v] < 0 || membership[v] >= n) {
            rc = ORC_BAD_ARG;
            goto done;
        }
    int64_t m2 = 0;
    for (int it = 0; it < n_iter; ++it) {
        ld_graph g = g0;   /* level 0 borrows the input graph */
        int own = 0;       /* g owns its arrays from level 1 on */
        for (int64_t v = 0; v < n; ++v) {
            top[v] = (int32_t)v;   /* node of v at the current level */
            comm[v] = membership[v];
        }
        ld_canon(n, comm, next);
        int level = 0;
        for (; level < max_levels; ++level) {
            const int64_t nv = g.nv;
            m2 = 0;
            for (int64_t v = 0; v < nv; ++v) {
                int64_t w = 0;
                for (int64_t e = g.ip[v]; e < g.ip[v + 1]; ++e) w += g.wt[e];
                k[v] = w;
                m2 += w;
            }
            if (m2 == 0) break;
            ld_move(&g, k, m2, G, max_rounds, comm, tot, s, touched, next);
            int64_t ncomm = 0;
            for (int64_t v = 0; v < nv; ++v) ncomm += comm[v] == v;
            if (ncomm == nv) break;   /* every community is a single node */
            ld_refine(&g, k, m2, G, max_rounds, comm, tot, ref, s, touched, target, wC, rtot, ext, size, picked,
                      next);
            ld_graph h = {0, NULL, NULL, NULL};
            int64_t *acc = (int64_t *)calloc((size_t)nv, sizeof(int64_t));
            if (!acc) {
                rc = ORC_NO_MEM;
                break;
            }
            const int64_t K = ld_aggregate(&g, ref, node, &h, acc, touched);
            free(acc);
            if (K == 0) {
                ld_free(&h);
                rc = ORC_NO_MEM;
                break;
            }
            if (K == nv) {   /* the refinement merged nothing */
                ld_free(&h);
                break;
            }
            /* the aggregate's communities: node of each community's smallest member */
            for (int64_t v = 0; v < nv; ++v) next[node[v]] = node[comm[v]];
            for (int64_t v = 0; v < n; ++v) top[v] = node[top[v]];
            if (own) ld_free(&g);
            g = h;
            own = 1;
            memcpy(comm, next, sizeof(int32_t) * (size_t)K);
        }
        for (int64_t v = 0; v < n; ++v) membership[v] = comm[top[v]];
        if (own) ld_free(&g);
        if (levels_run) *levels_run = level;
        if (rc != ORC_OK) goto done;
    }
    /* number by first appearance; quality on the input graph */
    {
        for (int64_t v = 0; v < n; ++v) next[v] = -1;
        int32_t K = 0;
        for (int64_t v = 0; v < n; ++v) {
            if (next[membership[v]] < 0) next[membership[v]] = K++;
            membership[v] = next[membership[v]];
        }
        if (n_comm) *n_comm = K;
        if (quality) {
            for (int64_t c = 0; c < K; ++c) {
                tot[c] = 0;
                rtot[c] = 0;
            }
            int64_t M = 0;
            for (int64_t v = 0; v < n; ++v)
                for (int64_t e = g0.ip[v]; e < g0.ip[v + 1]; ++e) {
                    tot[membership[v]] += g0.wt[e];
                    M += g0.wt[e];
                    if (membership[g0.col[e]] == membership[v]) rtot[membership[v]] += g0.wt[e];
                }
            double q = 0.0;
            for (int64_t c = 0; c < K && M > 0; ++c) {
                const double f = (double)tot[c] / (double)M;
                q += (double)rtot[c] / (double)M - gamma * f * f;
            }
            *quality = q;
        }
    }
done:
    ld_free(&g0);
    free(k); free(tot); free(s); free(wC); free(rtot); free(ext); free(comm); free(next); free(touched);
    free(ref); free(target); free(size); free(node); free(top); free(picked);
    return rc;
}
