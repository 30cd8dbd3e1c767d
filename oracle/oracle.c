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
