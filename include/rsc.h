/*
 * rsc.h -- C ABI of the GB300 neighbourhood-graph library.
 *
 * The library computes the neighbourhood-graph step of a scanpy-style
 * single-cell workflow on one GPU:
 *   1. exact k-nearest neighbours of every cell over its principal
 *      components (Euclidean or cosine distance; paper, Methods, "Custom GPU
 *      kernels", which defines the two distances, and "Dimensionality
 *      reduction and graph analysis", where the kNN graph feeds UMAP and
 *      Leiden), and
 *   2. the fuzzy connectivities graph built from those lists: per-cell rho and
 *      sigma of the smooth-kNN equation, directed weights, and the union
 *      G = A + A^T - A o A^T stored as CSR (paper, Methods,
 *      "Implementation": results follow scanpy, whose neighbours step builds
 *      this graph; "Dimensionality reduction and graph analysis": the graph is
 *      stored in .obsp for UMAP and Leiden).
 *
 * Conventions shared by every entry point
 *   - Every array argument is a DEVICE pointer owned by the caller, unless the
 *     argument's comment says "host".  Matrices are row-major and contiguous.
 *   - The library allocates no device memory: each call that needs scratch
 *     space takes a caller-provided `workspace` whose minimum size the matching
 *     *_workspace_size() returns.  Workspace pointers must be 256-byte aligned.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless documented otherwise.  Argument errors are found
 *     on the host before anything is launched.
 *   - Errors: a non-zero rsc_status is returned and rsc_last_error() gives a
 *     thread-local message.  Outputs are unspecified after an error.
 *   - Bounded waits: kernels that wait on in-kernel barriers give up after a
 *     fixed budget and record RSC_ERR_TIMEOUT in the workspace's status word;
 *     rsc_workspace_status() reads it back (it synchronises the stream).
 *   - Indices are int32 (n < 2^31 rows); CSR row pointers are int64.
 */
#ifndef RSC_H
#define RSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RSC_OK = 0,
    RSC_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or option        */
    RSC_ERR_CUDA = 2,          /* a CUDA runtime/driver call failed             */
    RSC_ERR_WORKSPACE = 3,     /* workspace missing or smaller than required    */
    RSC_ERR_TIMEOUT = 4,       /* an in-kernel wait exceeded its budget         */
    RSC_ERR_UNSUPPORTED = 5,   /* valid request this library does not implement */
    RSC_ERR_CAPACITY = 6       /* CSR output capacity smaller than nnz          */
} rsc_status;

typedef enum {
    RSC_EUCLIDEAN = 0,         /* sqrt(sum_t (x_t - y_t)^2)                      */
    RSC_COSINE = 1             /* 1 - x.y / (|x| |y|); 0 between two all-zero
                                  rows, 1 between an all-zero row and any other */
} rsc_metric;

typedef enum {
    RSC_FP32 = 0,              /* FP32 SIMT distances for candidate selection   */
    RSC_BF16 = 1,              /* BF16 tcgen05 tensor-core distances (FP32
                                  accumulate) for candidate selection            */
    RSC_FP8 = 3                /* FP8 E4M3 tcgen05 tensor-core distances (FP32
                                  accumulate; rows scaled by one power of two
                                  per call): half the operand bytes and MMA
                                  time of BF16, 3 mantissa bits, so long
                                  candidate lists (default 8k, at most 128);
                                  full scan only (no tile pruning); d <= 59
                                  (Euclidean) or 63 (cosine).  (Value 2 is
                                  reserved.)                                    */
} rsc_precision;

/* Options of rsc_knn.  Zero-initialise and set what you need. */
typedef struct {
    int32_t precision;   /* rsc_precision used to select candidates          */
    int32_t candidates;  /* candidates kept per query before the exact FP32
                            re-rank; 0 = default (k + 8 for FP32, 2k for BF16
                            Euclidean, 4k for BF16 cosine, 8k for FP8, at
                            most 64 / 128);
                            rounded up to a supported width (16, 32, 64)  */
    int32_t db_splits;   /* split the database into this many ranges handled
                            by separate CTAs (small n); 0 = automatic          */
    int32_t tc_parts;    /* tensor-core path: threads (column parts) per query
                            row, 2 or 4; 0 = automatic                          */
    void *stream;        /* cudaStream_t                                        */
    void *phase_events;  /* optional host array of 4 cudaEvent_t owned by the
                            caller, recorded on `stream` before the prep pass,
                            before the candidate search, before the exact
                            re-rank and after it (per-phase timing); NULL = off */
    int32_t locality;    /* tensor-core path: group rows by a coarse k-means
                            before the search and let every query tile scan its
                            own neighbourhood first (fewer top-k updates; the
                            result is unchanged).  0 = automatic (on for
                            n >= 16384), 1 = off, 2 = on                        */
    int32_t prune;       /* tensor-core path with locality ordering: after a first
                            pass over each query tile's neighbourhood, skip the
                            database tiles whose bounding sphere is provably too
                            far from the query tile's to improve any of its
                            lists (exact: the candidates equal the full scan's).
                            0 = automatic (on with the ordering, one database
                            split, d + 3 <= 64), 1 = off, 2 = on               */
    int32_t stages;      /* tensor-core path: shared-memory stages of the
                            database-tile pipeline, 2 .. 6 (clamped to what the
                            list shape's shared memory holds); 0 = automatic
                            (as many as fit, or the autotuner's choice)        */
} rsc_knn_opts;

/* Library version string (static storage). */
const char *rsc_version(void);

/* Thread-local message describing the last error returned on this thread. */
const char *rsc_last_error(void);

/*
 * Budget, in SM clock cycles, of every bounded wait inside the tensor-core
 * kernels (the barrier waits of the TMA producer, the MMA issuer and the
 * epilogue); 0 restores the default of about 1 s.  A diagnostic for
 * exercising the timeout path (the paper has no counterpart): with a budget
 * of a few hundred cycles the first wait of a search gives up, the kernel
 * records RSC_ERR_TIMEOUT in the workspace status word, lets its in-flight
 * copies and MMAs finish (those drains keep the default budget), frees its
 * tensor memory and returns; the outputs of that call are unspecified and
 * the next call with the default budget runs normally.  Process-wide;
 * applies to launches issued after the call.  Errors: RSC_ERR_INVALID_ARG
 * for a negative budget.
 */
rsc_status rsc_set_wait_budget(int64_t clocks);

/*
 * Reads and clears the status word that kernels write into `workspace`
 * (first 4 bytes).  Synchronises `stream`.  Returns RSC_OK when no kernel
 * recorded a failure, else the recorded rsc_status.
 */
rsc_status rsc_workspace_status(void *workspace, void *stream);

/*
 * Minimum workspace for rsc_knn with these arguments (host query; no GPU
 * work).  `opts` may be NULL (defaults).  Result in *bytes (host).
 */
rsc_status rsc_knn_workspace_size(int64_t n, int32_t d, int32_t k, int32_t metric,
                                  const rsc_knn_opts *opts, size_t *bytes);

/*
 * Exact k-nearest neighbours of every row of X among all rows of X.
 *   X        [n, d] float32 cells x principal components.
 *   n, d     1 <= n < 2^31, 1 <= d <= 64.
 *   k        1 <= k <= min(n, 64); for RSC_BF16 also 2k <= 64 by default.
 *   metric   rsc_metric.
 *   idx      [n, k] int32 out: neighbour row ids, self included, ordered by
 *            (distance, id) ascending.
 *   dist     [n, k] float32 out: Euclidean distance (not squared) or 1 - cos.
 * Method: candidates are selected with the precision in opts (FP32 SIMT or
 * BF16 tensor cores, the n x n distance matrix is never stored), then every
 * candidate is re-scored exactly in FP32 by direct difference and the k best
 * are kept.  Ties in the final order are broken by ascending id.
 */
rsc_status rsc_knn(const float *X, int64_t n, int32_t d, int32_t k, int32_t metric,
                   int32_t *idx, float *dist, const rsc_knn_opts *opts,
                   void *workspace, size_t workspace_bytes);

/*
 * Work done by the candidate search of the last rsc_knn call that used
 * `workspace` with these same arguments (a diagnostic; the paper has no
 * counterpart).  Counts pairs of a 128-row query tile and a 256-row database
 * tile: *pairs_total (host) = query tiles x database tiles, *pairs_scanned
 * (host) = the pairs whose distances were computed (= total without
 * pruning).  Reads the workspace after synchronising opts->stream.
 * Errors: RSC_ERR_INVALID_ARG for NULL outputs or arguments rsc_knn would
 * reject; RSC_ERR_WORKSPACE when the workspace is missing or too small.
 */
rsc_status rsc_knn_scan_stats(int64_t n, int32_t d, int32_t k, int32_t metric, const rsc_knn_opts *opts,
                              void *workspace, size_t workspace_bytes, int64_t *pairs_scanned,
                              int64_t *pairs_total);

/*
 * Autotuner.  Options left at 0 (db_splits, candidates, tc_parts) are
 * "automatic": rsc_knn and rsc_knn_batched then look up a process-wide table
 * of tuned choices keyed by (entry point, precision, metric, d, k, k_cross,
 * floor(log2 n)), and fall back to built-in defaults when it has no entry.
 * The rsc_autotune_* calls fill that table by timing candidate
 * configurations on the caller's own data with CUDA events on opts->stream,
 * by coordinate descent: database splits x column parts per row (list
 * shapes 2 x 16 and 4 x 16 for k <= 16), then the pipeline stages (3, 4, 5
 * and as many as fit), then candidate lists twice the default length; every
 * configuration returns exact FP32 distances of candidate sets at least as
 * large as the default's, so the choice never lowers recall.  The 128 x 256
 * tile (one M = 128 accumulator per query tile, N = 256 database rows per
 * MMA) is fixed: the pruning geometry, the batched work tables and the
 * TMEM double buffer (2 x 256 of the 512 columns) are built on it.
 * They synchronise the stream and leave the result of the last timed run in
 * the output arrays.
 */

/* Workspace large enough for every configuration rsc_autotune_knn tries. */
rsc_status rsc_autotune_workspace_size(int64_t n, int32_t d, int32_t k, int32_t metric,
                                       int32_t precision, size_t *bytes);

/*
 * Tune rsc_knn for (n, d, k, metric, opts->precision): `trials` timed runs
 * per configuration (>= 1).  On return *best (host) holds the chosen options
 * (stream and precision copied from opts) and *best_ms (host, may be NULL)
 * its time; the choice is stored in the table.
 */
rsc_status rsc_autotune_knn(const float *X, int64_t n, int32_t d, int32_t k, int32_t metric,
                            const rsc_knn_opts *opts, int32_t trials, int32_t *idx, float *dist,
                            rsc_knn_opts *best, float *best_ms, void *workspace,
                            size_t workspace_bytes);

/*
 * Tune rsc_knn_batched (column parts per row) the same way; the workspace is
 * sized by rsc_knn_batched_workspace_size with automatic options.
 */
rsc_status rsc_autotune_knn_batched(const float *X, int64_t n, int32_t d,
                                    const int64_t *sample_offsets, int32_t n_samples,
                                    int32_t k_within, int32_t k_cross, int32_t metric,
                                    const rsc_knn_opts *opts, int32_t trials,
                                    int32_t *idx_within, float *dist_within, int32_t *idx_cross,
                                    float *dist_cross, rsc_knn_opts *best, float *best_ms,
                                    void *workspace, size_t workspace_bytes);

/* Persist / restore / empty the tuned table (plain text, one entry per line;
 * host only). */
rsc_status rsc_autotune_save(const char *path);
rsc_status rsc_autotune_load(const char *path);
rsc_status rsc_autotune_clear(void);

/*
 * Minimum workspace for rsc_knn_batched (host query; no GPU work).
 */
rsc_status rsc_knn_batched_workspace_size(int64_t n, int32_t d, const int64_t *sample_offsets,
                                          int32_t n_samples, int32_t k_within, int32_t k_cross,
                                          int32_t metric, const rsc_knn_opts *opts, size_t *bytes);

/*
 * Batched exact kNN over samples (for batch-aware graphs).
 *   X               [n, d] float32; the cells of sample s are rows
 *                   sample_offsets[s] .. sample_offsets[s+1]-1.
 *   sample_offsets  HOST array of n_samples + 1 ascending int64, [0] = 0,
 *                   [n_samples] = n; every sample needs >= k_within cells.
 *   k_within        1 <= k_within <= 16: neighbours inside the cell's own
 *                   sample (self included).
 *   k_cross         1 <= k_cross <= min(4, k_within): neighbours taken from
 *                   EVERY sample, own sample included.
 *   idx_within, dist_within  [n, k_within] out, as rsc_knn restricted to the
 *                   cell's sample (global row ids, ordered by (distance, id)).
 *   idx_cross, dist_cross    [n, n_samples * k_cross] out: the k_cross nearest
 *                   cells of each sample, the whole row ordered by
 *                   (distance, id); n_samples * k_cross <= 1024.
 * Candidates come from one persistent BF16 tensor-core launch over
 * (query tile, sample) work items and are re-scored exactly in FP32 (the
 * precision option must be RSC_BF16).  With a non-NULL stream the launch
 * sequence is captured once into a CUDA graph (cached per argument set, up
 * to 8 entries per process) and replayed; the first call for an argument set
 * synchronises the stream.  d + 3 <= 64 (Euclidean) or d + 1 <= 64 (cosine).
 * Paper: per-group kernels over category offsets (Methods, "Perturbation
 * distance computation"); kNN graph construction (Methods, "Dimensionality
 * reduction and graph analysis").
 */
rsc_status rsc_knn_batched(const float *X, int64_t n, int32_t d, const int64_t *sample_offsets,
                           int32_t n_samples, int32_t k_within, int32_t k_cross, int32_t metric,
                           int32_t *idx_within, float *dist_within, int32_t *idx_cross,
                           float *dist_cross, const rsc_knn_opts *opts, void *workspace,
                           size_t workspace_bytes);

/*
 * Work done by the last rsc_knn_batched on `workspace` with these same
 * arguments (a diagnostic; the paper has no counterpart).  Counts pairs of a
 * 128-row query tile and a 256-row database tile of one sample:
 * *pairs_total (host) = query tiles x all samples' database tiles,
 * *pairs_scanned (host) = the pairs whose distances were computed (= total
 * without pruning).  Reads the workspace after synchronising opts->stream.
 * Errors: RSC_ERR_INVALID_ARG for NULL outputs or arguments rsc_knn_batched
 * would reject; RSC_ERR_WORKSPACE when the workspace is missing or too small.
 */
rsc_status rsc_knn_batched_scan_stats(int64_t n, int32_t d, const int64_t *sample_offsets, int32_t n_samples,
                                      int32_t k_within, int32_t k_cross, int32_t metric,
                                      const rsc_knn_opts *opts, void *workspace, size_t workspace_bytes,
                                      int64_t *pairs_scanned, int64_t *pairs_total);

/*
 * Learned partitioner (candidate pruning for the exact search).
 *
 * A handle owns a small network d -> hidden -> hidden -> n_parts (ReLU; FP32
 * master weights, bfloat16-rounded weights and activations in every GEMM when
 * bf16_weights != 0, FP32 accumulation), n_parts k-means centroids and, once
 * built, an index of one database: its rows counting-sorted by the part the
 * network ranks first.  The handle is the one object of this library that
 * allocates device memory (create, build_index); destroy frees it.
 * rsc_knn_partitioned answers a query by scanning only the n_probe parts the
 * network ranks highest (or, with routing = 1, the n_probe nearest centroids:
 * the same parts and budget without the network), scoring candidates with
 * the BF16 tensor-core search and re-scoring them exactly in FP32: the result
 * is exact inside the probed parts and approximate overall (recall < 1).
 * The paper does not describe this component; its kNN is cuVS on the GPU and
 * PyNNDescent on the CPU (Methods, "Benchmarking").  Euclidean only, k <= 16,
 * d <= 61, n_parts in [8, 1024], hidden in [8, 1024].
 */
typedef struct rsc_partitioner rsc_partitioner;

rsc_status rsc_partitioner_create(int32_t d, int32_t n_parts, int32_t hidden, int32_t bf16_weights,
                                  uint64_t seed, rsc_partitioner **out);
rsc_status rsc_partitioner_destroy(rsc_partitioner *p);

/* Network parameters as one FP32 host array [W1 (hidden x d), b1, W2 (hidden x
 * hidden), b2, W3 (n_parts x hidden), b3], weights row-major out x in. */
rsc_status rsc_partitioner_param_count(const rsc_partitioner *p, int64_t *count);
rsc_status rsc_partitioner_get_params(const rsc_partitioner *p, float *host_out);
rsc_status rsc_partitioner_set_params(rsc_partitioner *p, const float *host_in);   /* resets Adam */

/*
 * Soft-target cross-entropy of a batch and its gradient (one forward and
 * backward pass of the training kernels, no update): loss = mean over rows of
 * -sum_p T[b, p] log softmax(z_b)_p.  Xb [batch, d], T [batch, n_parts] and
 * grad [param_count] are device arrays (grad may be NULL); *loss_host is
 * written after synchronising the stream.
 */
rsc_status rsc_partitioner_loss_grad_workspace_size(const rsc_partitioner *p, int32_t batch, size_t *bytes);
rsc_status rsc_partitioner_loss_grad(rsc_partitioner *p, const float *Xb, const float *T, int32_t batch,
                                     float *loss_host, float *grad, void *workspace,
                                     size_t workspace_bytes, void *stream);

/* Workspace for build_index / train (n_train rows, k) / rsc_knn_partitioned
 * (n_queries, n_probe); pass 0 for what a call does not use. */
rsc_status rsc_partitioner_workspace_size(const rsc_partitioner *p, int64_t n, int64_t n_train,
                                          int32_t k, int64_t n_queries, int32_t n_probe,
                                          size_t *bytes);

/*
 * Fit the partitioner on X [n, d] (device) and index X:
 *   1. k-means (kmeans_iters Lloyd steps) on the training rows train_rows
 *      (device int32 [n_train], n_parts <= n_train <= n; initial centroids =
 *      the first n_parts training rows); every row's label = nearest centroid;
 *   2. exact k nearest neighbours of each training row among all n rows;
 *   3. `epochs` passes of minibatch Adam (lr; betas 0.9, 0.999; eps 1e-8) on
 *      the soft target "histogram of the labels of my k neighbours";
 *   4. rsc_partitioner_build_index(X).
 * Synchronises the stream; *final_loss (host, nullable) = last epoch's loss.
 */
rsc_status rsc_partitioner_train(rsc_partitioner *p, const float *X, int64_t n,
                                 const int32_t *train_rows, int64_t n_train, int32_t k,
                                 int32_t kmeans_iters, int32_t epochs, int32_t batch, float lr,
                                 float *final_loss, void *workspace, size_t workspace_bytes,
                                 void *stream);

/* Assign every row of X to its network top-1 part and sort (re-allocates the
 * handle's index when n changes). */
rsc_status rsc_partitioner_build_index(rsc_partitioner *p, const float *X, int64_t n,
                                       void *workspace, size_t workspace_bytes, void *stream);

/*
 * k nearest neighbours (Euclidean, ids of X, self included when probed,
 * ordered by (distance, id)) of query_rows (device int32 [n_queries]; NULL =
 * every row, n_queries ignored) among the rows of the indexed X, probing
 * n_probe in {1, 2, 4, 8} parts per query.  routing: 0 = the network's
 * top parts, 1 = nearest centroids.  idx/dist [n_queries, k].
 */
rsc_status rsc_knn_partitioned(rsc_partitioner *p, const float *X, int64_t n, int32_t k,
                               int32_t n_probe, int32_t routing, const int32_t *query_rows,
                               int64_t n_queries, int32_t *idx, float *dist, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Network parameters and centroids to / from a binary file (host only; the
 * index is rebuilt with build_index after loading). */
rsc_status rsc_partitioner_save(const rsc_partitioner *p, const char *path);
rsc_status rsc_partitioner_load(const char *path, rsc_partitioner **out);

/*
 * Minimum workspace for rsc_connectivities / rsc_connectivities_nnz.
 */
rsc_status rsc_connectivities_workspace_size(int64_t n, int32_t k, size_t *bytes);

/*
 * Upper bound on the number of stored entries of the connectivities graph:
 * 2 * n * (k - 1) (every directed non-self edge stored twice).
 */
int64_t rsc_connectivities_max_nnz(int64_t n, int32_t k);

/*
 * Fuzzy connectivities of a kNN graph (UMAP smooth-kNN + fuzzy union).
 *   idx, dist  [n, k] as returned by rsc_knn (each row ascending by
 *              distance, distinct ids per row; slots with idx < 0 or >= n
 *              are ignored).  1 <= k <= 256 (with k = 1 every row lists only
 *              itself and the graph is empty).
 *   indptr     [n + 1] int64 out; indptr[n] = nnz.
 *   indices    [nnz_capacity] int32 out, ascending within each row.
 *   data       [nnz_capacity] float32 out.
 *   rho, sigma [n] float32 out, or NULL.
 * Per row i: rho_i = first non-zero distance; sigma_i solves
 *   sum_{c=1}^{k-1} exp(-max(0, d_ic - rho_i) / sigma_i) = log2(k)
 * by at most 64 bisection steps (stop within 1e-5), then is floored at
 * 1e-3 * mean row distance (1e-3 * mean of all distances when rho_i = 0);
 * w_ic = 0 for the row itself, 1 when d_ic <= rho_i, else
 * exp(-(d_ic - rho_i) / sigma_i).  G = A + A^T - A o A^T without the diagonal
 * or zeros.  All arithmetic is FP32.
 * If nnz_capacity >= rsc_connectivities_max_nnz(n, k) the call is
 * asynchronous; otherwise it synchronises once to compare nnz with the
 * capacity and returns RSC_ERR_CAPACITY (indptr valid) when it does not fit.
 */
rsc_status rsc_connectivities(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                              int64_t *indptr, int32_t *indices, float *data,
                              int64_t nnz_capacity, float *rho, float *sigma,
                              void *workspace, size_t workspace_bytes, void *stream);

/*
 * rsc_connectivities without a caller workspace and without allocating.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot hand out device memory when they build the graph, such as a host
 * application whose own pool has reserved the device's memory and offers
 * plug-ins no allocation hook, or a service with a fixed device-memory budget
 * that may not grow after start-up.  Same arguments and results as
 * rsc_connectivities, except:
 *   - scratch comes from a 32 MiB array declared by the library (held by
 *     every GPU that loads the library until the process exits); problems
 *     whose rsc_connectivities_workspace_size(n, k) exceeds 32 MiB are
 *     rejected with RSC_ERR_WORKSPACE before any GPU work (about 700 bytes
 *     per row at k = 15: up to 47,932 rows; up to 40,520 rows at k = 30);
 *   - nnz_capacity must be at least rsc_connectivities_max_nnz(n, k), so the
 *     call never synchronises to check the size;
 *   - every call looks up the array's device address in the calling thread's
 *     current context (a host query, no GPU work), so the call stays valid
 *     after cudaDeviceReset or under a context the caller made current.
 * All calls share the one array, which keeps the last call's contents (the
 * call clears what must start at zero): calls whose work overlaps on the GPU
 * (on different streams, or from different host threads) race and corrupt
 * each other's results.  Issue them on one stream, or order them.  The call
 * itself calls no cudaMalloc, cudaFree or other allocating routine.
 */
rsc_status rsc_connectivities_static(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                                     int64_t *indptr, int32_t *indices, float *data,
                                     int64_t nnz_capacity, float *rho, float *sigma, void *stream);

/*
 * Number of stored entries rsc_connectivities would produce, written to
 * *nnz (host).  Synchronises `stream`.
 */
rsc_status rsc_connectivities_nnz(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                                  int64_t *nnz, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* ------------------------------------------------------------ UMAP layout
 *
 * The layout step UMAP runs on the neighbourhood graph (paper, Methods,
 * "Dimensionality reduction and graph analysis": UMAP on the stored graph),
 * by the UMAP method's edge-sampled stochastic gradient optimisation
 * (McInnes, Healy & Melville 2018, "Optimizing the embedding").
 */
typedef struct {
    float a, b;                    /* phi(d) = 1 / (1 + a d^(2b)) (rsc_umap_find_ab) */
    float gamma;                   /* repulsion strength (1)                          */
    float learning_rate;           /* alpha of the first epoch (1)                    */
    int32_t negative_sample_rate;  /* negatives drawn per sampled entry (5)           */
    int32_t n_epochs;              /* N, length of the schedule (200; 500 at <= 10,000
                                      cells in scanpy)                                */
    int32_t epoch_first;           /* first epoch run, 1-based (0: 1)                 */
    int32_t epoch_last;            /* last epoch run, inclusive (0: N)                */
    uint64_t seed;                 /* negative-sample generator seed                  */
    void *stream;                  /* cudaStream_t, NULL = legacy default stream      */
} rsc_umap_opts;

/*
 * a and b of phi(d) = 1 / (1 + a d^(2b)) fitted by least squares to the
 * target curve 1 for d < min_dist, exp(-(d - min_dist) / spread) beyond, on
 * 300 evenly spaced points of [0, 3 spread] (the UMAP method's choice of
 * a, b from spread and min_dist).  Host only; Levenberg-Marquardt from
 * a = b = 1.  scanpy's defaults (spread 1, min_dist 0.5) give a = 0.583,
 * b = 1.334.  Errors: RSC_ERR_INVALID_ARG for NULL outputs, spread <= 0,
 * min_dist < 0 or a fit that does not converge.
 */
rsc_status rsc_umap_find_ab(float spread, float min_dist, float *a, float *b);

/*
 * Minimum workspace for rsc_umap_layout: two [n, dim] position buffers (rows
 * padded to 4 floats when dim = 3), the entries' sampling frequencies [nnz]
 * and the largest weight.
 */
rsc_status rsc_umap_workspace_size(int64_t n, int64_t nnz, int32_t dim, size_t *bytes);

/*
 * Epochs opts->epoch_first .. opts->epoch_last of the N-epoch UMAP layout of a
 * graph, in place on `embedding`.
 *   indptr [n + 1] int64, indices [nnz] int32, data [nnz] float32: the graph
 *              as CSR (rsc_connectivities' output).  It must be symmetric
 *              with equal values (G_ij == G_ji bit for bit, both entries
 *              stored), as the fuzzy union is: each vertex gathers the moves
 *              of its own row, which equal the per-entry moves only then.
 *   embedding  [n, dim] float32 row-major, 1 <= dim <= 4: the positions the
 *              epochs start from (an initial layout), replaced by the
 *              positions after the last epoch run.
 * Epoch n (alpha_n = learning_rate (1 - (n - 1) / N)) samples entry e of
 * weight w_e when floor(n f_e) > floor((n - 1) f_e), f_e = w_e / max w, both
 * in FP32, so entry e is sampled floor(N f_e) times in N epochs.  A sampled
 * entry i -> j moves i by 2 alpha clip(c (y_i - y_j)) with
 * c = -2ab d^(2(b-1)) / (1 + a d^(2b)) (its own pull and that of its mirror
 * j -> i), then draws negative_sample_rate vertices v: negative q is vertex
 * h * n >> 32, h the high (q even) or low (q odd) 32 bits of output number
 * ((n - 1) nnz + e) ceil(r / 2) + floor(q / 2) + 1 of SplitMix64 seeded with
 * `seed` (r = negative_sample_rate), and moves i by
 * alpha clip(c' (y_i - y_v)), c' = 2 gamma b / ((0.001 + d^2)(1 + a d^(2b))).
 * clip() bounds each coordinate to [-4, 4]; a zero distance moves nothing.
 * Every epoch reads the positions the previous one wrote, and all moves of an
 * epoch are summed (FP32, a fixed order per vertex): the result is
 * deterministic, and running epochs 1..m and then m+1..N gives the same
 * positions as one call.  Asynchronous on opts->stream.
 * Errors: RSC_ERR_INVALID_ARG for NULL pointers, n < 1, n >= 2^31, nnz < 0,
 * nnz >= 2^31, dim outside 1..4, n_epochs outside 1..100,000, an epoch range
 * outside 1..N, negative_sample_rate outside 0..64 or non-finite a, b, gamma
 * or learning_rate; RSC_ERR_WORKSPACE when the workspace is too small.  An
 * indptr that is not monotone within [0, nnz], or a sampled column outside
 * [0, n), is skipped and recorded as RSC_ERR_INVALID_ARG in the workspace
 * status word (rsc_workspace_status); nothing is read out of bounds.
 */
rsc_status rsc_umap_layout(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n,
                           int64_t nnz, int32_t dim, float *embedding, const rsc_umap_opts *opts,
                           void *workspace, size_t workspace_bytes);

/* ------------------------------------------------------------- E-distance
 *
 * Energy distance between groups of cells (paper, Methods, "Perturbation
 * distance computation"): E(a, b) = 2 d(a, b) - d(a, a) - d(b, b), d the mean
 * Euclidean distance between the cells of a and b (a != b: all n_a n_b pairs;
 * a == b: the n_a (n_a - 1) / 2 pairs i < j, 0 for a group of fewer than two
 * cells).  Groups are CSR-style: group g holds the cells
 * cell_index[group_offsets[g] .. group_offsets[g + 1]) (the paper's category
 * offsets and sorted cell index; cell_index NULL: rows group_offsets[g] ..
 * group_offsets[g + 1] of X themselves).
 */

/*
 * Minimum workspace for rsc_edistance with these groups and pairs (host-only
 * query).  group_offsets and pairs are host arrays, as in rsc_edistance.
 */
rsc_status rsc_edistance_workspace_size(int64_t n_rows, int32_t d, const int64_t *group_offsets, int32_t n_groups,
                                        const int32_t *pairs, int64_t n_pairs, size_t *bytes);

/*
 * Distance sums, mean distances and energy distances of group pairs.
 *   X             [n_rows, d] float32 row-major (device), 1 <= d <= 58
 *                 (RSC_ERR_UNSUPPORTED above: the three K blocks hold d + 6
 *                 columns each).
 *   cell_index    [group_offsets[G]] int32 device row ids, or NULL.
 *   group_offsets [G + 1] int64 HOST array, group_offsets[0] = 0,
 *                 non-decreasing, group_offsets[G] < 2^31; 1 <= G <= 65535.
 *   pairs         [n_pairs, 2] int32 HOST array of requested pairs (a, b),
 *                 a <= b (duplicates allowed), or NULL for every pair a <= b;
 *                 explicit pairs need G <= 16384.  The paper's
 *                 onesided_distances is the pairs (ref, b) and (b, b).
 *   sums          [G, G] float64 device out: S[a][b] (a <= b) for the
 *                 requested pairs, the sum of the pair's distances (upper
 *                 triangle of the group on the diagonal); every other entry 0.
 *   mean, E       [G, G] float64 device out, or NULL: for every (a, b) (both
 *                 orders) whose pair was requested, the mean distance, and the
 *                 energy distance where the pair and both diagonals were
 *                 requested; NaN elsewhere.
 * Distances are computed on tensor cores from BF16 operands split into high
 * and low parts (three products per coordinate pair, FP32 accumulation, each
 * row centred on a common point first), summed in FP32 per 32 columns and in
 * float-float pairs (about 48 significant bits) beyond, each pair's two parts
 * added to the FP64 sums by atomics; expect about 1e-6 relative error in the
 * sums.  Asynchronous on
 * `stream`, except that the offsets, the work list and the pair mask are copied
 * from host memory before the call returns.  Errors: RSC_ERR_INVALID_ARG for
 * NULL pointers, bad offsets, pairs out of range or a > b, n_rows outside
 * [1, 2^31) or cells beyond n_rows without a cell index; RSC_ERR_WORKSPACE
 * when the workspace is missing or small.  A cell index outside [0, n_rows)
 * is recorded as RSC_ERR_INVALID_ARG in the workspace status word
 * (rsc_workspace_status); that cell then reads row 0.  Kernel waits that run
 * out their budget record RSC_ERR_TIMEOUT there.
 */
rsc_status rsc_edistance(const float *X, int64_t n_rows, int32_t d, const int32_t *cell_index,
                         const int64_t *group_offsets, int32_t n_groups, const int32_t *pairs, int64_t n_pairs,
                         double *sums, double *mean, double *E, void *workspace, size_t workspace_bytes,
                         void *stream);

/* ------------------------------------------------- approximate kNN (NN-descent)
 *
 * The paper's CPU neighbour search is PyNNDescent (Methods, "Benchmarking"), an
 * approximate kNN by NN-descent (Dong, Charikar & Li, WWW 2011: a neighbour of
 * a neighbour is probably a neighbour).  This is its synchronous form with
 * deterministic sampling, a third speed / recall point beside the exact
 * search.  Euclidean distance only.
 */
typedef struct {
    int32_t sample;      /* S: entries flagged new sampled per list and
                            iteration, 1 <= S <= k (0: k)                       */
    int32_t rev_slots;   /* R: reverse-sample slots per point, a power of two
                            in 1 .. 64 (0: 32)                                  */
    int32_t cand_slots;  /* C: candidate slots per point, a power of two in
                            1 .. 64 (0: 64)                                     */
    int32_t max_iters;   /* T: iterations at most, 1 .. 64 (0: max(5,
                            round(log2 n)), PyNNDescent's count)                 */
    double delta;        /* stop after an iteration that changed fewer than
                            delta n k list entries (0: run all T)               */
    uint64_t seed;       /* generator seed of the initial lists and the
                            reverse-sample priorities                           */
    void *stream;        /* cudaStream_t, NULL = legacy default stream          */
} rsc_nnd_opts;

/* Minimum workspace for rsc_knn_descent: the lists (8 n k bytes), two masks
 * per point, 2 n R + n C slots of 8 bytes, the change counters. */
rsc_status rsc_knn_descent_workspace_size(int64_t n, int32_t d, int32_t k, const rsc_nnd_opts *opts, size_t *bytes);

/*
 * Approximate k-nearest-neighbour lists of every row of X by NN-descent.
 *   X        [n, d] float32 row-major (device), 2 <= n < 2^31, d >= 1.
 *   init_idx [n, k] int32 (device) or NULL: lists to start from (for example
 *            an earlier graph); entries outside [0, n), repeats and the row
 *            itself are skipped, and hashed draws fill what is left.
 *   idx      [n, k] int32 out: each row's list, nearest first, the row itself
 *            included (k <= min(64, n)); dist [n, k] float32 out: Euclidean
 *            distance sqrtf(delta2) of each entry.
 *   changes  [64] int64 device out or NULL: list entries changed by
 *            iteration t (0 for iterations not run).
 * Definition (every step on FP32 squared distances delta2(a, b): acc = 0,
 * then acc = fmaf(x_a[t] - x_b[t], x_a[t] - x_b[t], acc) for t = 0 .. d-1;
 * lists ordered by key = bits(delta2) << 32 | id; G(i) = output i >= 1 of
 * SplitMix64 seeded with seed; slot_b(id) = (id * 0x9E3779B1 mod 2^32) >>
 * (32 - b), 0 for b = 0):
 *   initial list of u: u, then the valid new entries of init_idx[u] in
 *   order, then the new values of (u + 1 + G(2ku + j + 1) mod (n - 1)) mod n,
 *   j = 0 .. 2k-1, then u + 1, u + 2, ... mod n, each only while the list is
 *   short of k; all entries but u flagged new.
 *   Iteration t, on the lists as they were when it began:
 *   1. new_f(u) = the first S entries flagged new (u excluded), whose flags
 *      are cleared; old_f(u) = the entries flagged old before (u excluded).
 *   2. u offers key (G(((t+1) << 40) | u) >> 32) << 32 | u to slot
 *      slot_log2R(u) of the new (old) reverse slots of every w in new_f(u)
 *      (old_f(u)); a slot keeps its smallest key.
 *   3. new(v) = new_f(v) and v's new reverse ids; old(v) = old_f(v) and v's
 *      old reverse ids, minus new(v).
 *   4. For every v and pair {a, b}, a != b, a in new(v), b in new(v) or
 *      old(v): b is offered to a with key(delta2(a, b), b) if that is below
 *      the key of a's last entry, into slot slot_log2C(b) of a's C candidate
 *      slots (a slot keeps its smallest key); the same for a to b.
 *   5. Each list becomes the k smallest distinct keys of itself and its
 *      candidates; kept entries keep their flags, entered ones are new;
 *      changes[t] counts the entered ones.
 *   6. The run stops after an iteration with changes[t] < delta n k.
 * The result is deterministic (the same bits on every run and launch shape).
 * Asynchronous on opts->stream.  Errors: RSC_ERR_INVALID_ARG for NULL
 * pointers, sizes or options outside the ranges above; RSC_ERR_WORKSPACE for
 * a missing or small workspace; RSC_ERR_UNSUPPORTED when the join's shared
 * memory (4 d (S + 2R + k) bytes and a little more) exceeds 200 KiB.
 */
/*
 * Pairs joined by each iteration of the last rsc_knn_descent call that used
 * this workspace (a statistic for throughput accounting; the paper has no
 * counterpart): pairs[t] = sum over points v of a (a - 1) / 2 + a o, a and o
 * the sizes of v's new and old join lists.  pairs: HOST array of 64.
 * Synchronises the device.
 */
rsc_status rsc_knn_descent_pairs(const void *workspace, size_t workspace_bytes, int64_t *pairs);

rsc_status rsc_knn_descent(const float *X, int64_t n, int32_t d, int32_t k, const int32_t *init_idx, int32_t *idx,
                           float *dist, int64_t *changes, const rsc_nnd_opts *opts, void *workspace,
                           size_t workspace_bytes);

/* ---------------------------------------------------------------- Leiden
 *
 * Communities of the neighbourhood graph by the Leiden method (Traag, Waltman
 * & van Eck, Sci. Rep. 2019), the clustering the paper runs on the stored
 * graph (Methods, "Dimensionality reduction and graph analysis"), with the
 * modularity quality function and a resolution gamma, as scanpy calls it.
 */
typedef struct {
    double resolution;      /* gamma, in (0, 32768) (0: 1)                      */
    int32_t n_iterations;   /* whole Leiden runs, each from the previous
                               partition (0: 2, scanpy's count)                 */
    int32_t max_levels;     /* aggregation levels per run at most (0: 32)       */
    int32_t max_rounds;     /* rounds per moving or refinement phase (0: 8)     */
    void *stream;           /* cudaStream_t, NULL = legacy default stream       */
} rsc_leiden_opts;

/* Minimum workspace for rsc_leiden (host-only query): two copies of the graph
 * with 64-bit weights, hash tables of 4 nnz + 2 n slots (12 bytes each), a
 * few arrays of n. */
rsc_status rsc_leiden_workspace_size(int64_t n, int64_t nnz, size_t *bytes);

/*
 * Leiden communities of a graph.
 *   indptr [n + 1] int64, indices [nnz] int32, data [nnz] float32 (device):
 *              the graph as CSR, symmetric (rsc_connectivities' output);
 *              weights >= 0; a diagonal entry is a self-loop.
 *   init       [n] int32 (device) starting partition labels in [0, n), or NULL
 *              (every vertex alone).
 *   membership [n] int32 device out: each vertex's community, numbered
 *              0, 1, ... in order of first appearance over the vertices.
 *   n_communities, modularity: HOST out (nullable): the community count and
 *              sum_c (in_c / 2m - gamma (tot_c / 2m)^2) of the result.
 * Definition (every decision exact, on W = rint(w 2^32) as 64-bit integers
 * and G = rint(gamma 2^16); k_v = the row sum of W, 2m = sum of k, tot_c =
 * sum of k over c; labels are vertex ids and every phase ends by labelling a
 * community with its smallest member; s_c = the weight of v's entries with
 * W > 0 to other vertices of c):
 *   1. Moving, in rounds r = 0, 1, ... on the state of the round's start:
 *      v picks the neighbouring community c != a = comm(v) with the largest
 *      g(c) = s_c 2m 2^16 - G k_v tot_c (ties: smaller c) and moves there if
 *      g(c) > s_a 2m 2^16 - G k_v (tot_a - k_v) and c < a in even rounds,
 *      c > a in odd ones; until two rounds in a row move nothing, or
 *      max_rounds (8 by default: on kNN graphs of 60,000 to 1,000,000
 *      cells, 4 to 64 rounds give the same modularity within 1e-4).
 *   2. Refinement inside each community C: every vertex starts alone; a
 *      vertex still alone with s_{C-v} 2m 2^16 >= G k_v (tot_C - k_v) picks,
 *      among the subcommunities S of its neighbours in C with
 *      ext_S 2m 2^16 >= G tot_S (tot_C - tot_S) (ext_S: the weight from S to
 *      C - S), the one with the largest g(S) = s_S 2m 2^16 - G k_v tot_S >= 0
 *      (ties: smaller label); vertices nobody picked join their pick, all at
 *      once; until a round moves nothing, or max_rounds.  (The paper draws
 *      the pick at random with a probability growing with the gain; this is
 *      its limit without randomness.)
 *   3. Aggregation: one node per subcommunity, numbered by smallest member;
 *      node weights are sums of member weights (self-loops hold the internal
 *      weight); each node starts in its community of step 1.
 *   Levels repeat until step 1 leaves every community a single node, step 2
 *   merges nothing, or max_levels; n_iterations runs.
 * Deterministic: the same partition on every run (equal to the library's
 * CPU statement of the same steps).  Synchronous: the host drives the rounds
 * and reads each round's move count, so the call returns when the result is
 * ready.  Errors: RSC_ERR_INVALID_ARG for NULL pointers, n outside
 * [1, 2^31), options out of range, or (found on the device before any round)
 * row pointers or columns outside the graph or starting labels outside
 * [0, n); RSC_ERR_WORKSPACE for a missing or small workspace.
 */
/*
 * Work of the last successful rsc_leiden call made on this thread (a statistic
 * for throughput accounting; the paper has no counterpart).  stats: HOST
 * array of 6: levels run (over all runs), moving rounds, refinement rounds,
 * graph entries read by those rounds (a moving round reads every entry of its
 * level once, a refinement round twice), vertices visited likewise, and the
 * kernels launched.
 */
rsc_status rsc_leiden_last_stats(int64_t *stats);

rsc_status rsc_leiden(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n, int64_t nnz,
                      const int32_t *init, int32_t *membership, int64_t *n_communities, double *modularity,
                      const rsc_leiden_opts *opts, void *workspace, size_t workspace_bytes);

#ifdef __cplusplus
}
#endif

#endif /* RSC_H */
