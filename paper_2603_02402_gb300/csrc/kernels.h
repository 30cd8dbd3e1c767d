// Launchers of the library's kernels (internal; the public ABI is rsc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsc {

// ---- prep.cu --------------------------------------------------------------
// Y [n, DP] float32: the rows of X minus the column means (Euclidean) or
// X / |X| (cosine), zero padded to DP columns; for cosine, column d holds 1
// for an all-zero row.  ny [n]: sum_t Y_t^2 in FP32 (Euclidean) or 0 (cosine).
// scratch: prep_scratch_floats() floats.
size_t prep_scratch_floats();
cudaError_t launch_prep_fp32(const float *X, int64_t n, int d, int DP, int metric,
                             float *Y, float *ny, float *scratch, cudaStream_t st);

// ---- knn_simt.cu ----------------------------------------------------------
// FP32 SIMT candidate search: for every query row and database split s,
// cand[(s * n + q) * KC + c] = the KC columns with the smallest
// ny_j - 2 * Y_q . Y_j inside the split (ties keep the earlier column).
// Columns width .. DP - 1 of Y are zero (DP - 7 <= width <= DP).
bool knn_simt_supported(int DP, int KC);
cudaError_t launch_knn_simt(const float *Y, const float *ny, int64_t n, int DP, int width, int KC,
                            int splits, int64_t split_len, int32_t *cand, cudaStream_t st);

// ---- knn_tc.cu ------------------------------------------------------------
// BF16 tensor-core candidate search.  Qb/Db: [n, 64 * tc_kb(d, metric)] bf16
// operand rows built by launch_prep_bf16 from the FP32 prep rows Y.  Each
// row's candidates come in sh.parts lists of sh.list ids (one list per column
// part of the database tiles): cand holds splits * parts lists per query, list
// (s * parts + p) of query q at cand[((s * parts + p) * n + q) * list].
// Database splits must be multiples of knn_tc_split_align() rows.  Bounded
// waits record RSC_ERR_TIMEOUT in *status.
struct TcShape {
    int parts;        // lists per row and split (0: no kernel for this request)
    int list;         // ids per list
    int stages = 0;   // database-tile pipeline stages (0: as many as shared memory holds)
};
int tc_kb(int d, int metric);
TcShape knn_tc_shape(int d, int metric, int k, int want, int parts_req);
bool knn_tc_supported(int d, int metric);
int64_t knn_tc_split_align();
// perm (nullable): operand row i is built from Y row perm[i].
cudaError_t launch_prep_bf16(const float *Y, int64_t n, int d, int DP, int metric, const int32_t *perm, void *Qb,
                             void *Db, cudaStream_t st);
// window > 0: each query tile first scans the `window` database tiles on
// either side of its own position (rows in locality order), then the rest.
cudaError_t launch_knn_tc(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh, int splits,
                          int64_t split_len, int window, int32_t *cand, unsigned int *status, cudaStream_t st);

// ---- knn_tc_fp8.cu --------------------------------------------------------
// FP8 (E4M3) variant of the tensor-core search: Qf/Df [n, 64] bytes built by
// launch_prep_fp8 (one power-of-two scale per call from the largest |y|,
// written to *amax), full scan (window first on ordered rows), candidate
// lists as launch_knn_tc.
bool knn_tc_fp8_supported(int d, int metric);
cudaError_t launch_prep_fp8(const float *Y, int64_t n, int d, int DP, int metric, const int32_t *perm, void *Qf,
                            void *Df, unsigned int *amax, cudaStream_t st);
cudaError_t launch_knn_tc_fp8(const void *Qf, const void *Df, int64_t n, int d, int metric, TcShape sh, int splits,
                              int64_t split_len, int window, int32_t *cand, unsigned int *status, cudaStream_t st);

// ---- mlp_tc.cu ------------------------------------------------------------------
// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]) on the tensor cores (operands
// rounded to BF16, FP32 accumulation), A(m, k) = A[m*sam + k*sak], B(k, n) =
// B[k*sbk + n*sbn]; flags 4 / 8: ReLU on A / B as they are read.  Bounded
// waits record RSC_ERR_TIMEOUT in *status.
cudaError_t launch_tc_gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                           const float *B, int64_t sbk, int64_t sbn, float *C, int64_t ldc, const float *bias,
                           int flags, unsigned int *status);

// ---- order.cu -------------------------------------------------------------------
// Locality ordering: two-level k-means (C1 coarse clusters, then C2 sub-
// clusters inside each; Lloyd on strided samples), then a stable counting
// sort of all rows by (coarse, sub) label.
constexpr int kOrderSub = 16;           // sub-clusters per coarse cluster
constexpr int kOrderLeafRows = 512;     // target rows per sub-cluster
constexpr int kOrderMaxCoarse = 128;
constexpr int kOrderMaxLeaves = kOrderMaxCoarse * kOrderSub;
constexpr int kOrderIters = 2;
constexpr int64_t kOrderMinRows = 16384;   // automatic ordering from this many rows
constexpr int kOrderWindow = 2;            // database tiles on each side scanned first
struct OrderShape {
    int C1, C2;
    int64_t m1, step1, m2, step2;
    int nchunk;
};
OrderShape order_shape(int64_t n);
size_t order_scratch_bytes(int64_t n, int DP, int groups = 0);
// perm[sorted position] = original row, for the FP32 prep rows Y [n, DP].
// goff (device, [G + 1], nullable): row groups (samples) whose position
// ranges must be kept; each group's rows come out in cluster order.
cudaError_t launch_locality_order(const float *Y, int64_t n, int DP, int iters, int32_t *perm, void *scratch,
                                  cudaStream_t st, const int64_t *goff = nullptr, int G = 0);

// ---- knn_tc_prune.cu / prune.cu ---------------------------------------------------
// Pruned search on rows in locality order (one database split, KB = 1):
// a window pass saves every (row, part) list (keys and ids, [n, parts, list]),
// launch_prune_bounds keeps per query tile the database tiles that can still
// improve one of its lists, and the list pass resumes the lists over them.
constexpr int64_t kPruneListCap = int64_t(1) << 28;   // kept (query tile, tile) pairs stored at most
struct PruneShape {
    int qtiles, dtiles, nchunk;
    int64_t cap;
};
struct PruneOut {
    int64_t *tile_off;   // [qtiles + 1]
    int32_t *tiles;      // [cap]
    int32_t *order;      // [qtiles]: query tiles by decreasing kept-tile count (list pass item order)
    int32_t *overflow;   // [1]: more kept pairs than cap (the list pass then scans every tile)
    int32_t *counter;    // [1]: the list pass's dynamic item counter
};
PruneShape prune_shape(int64_t n, int BM, int BN);
size_t prune_scratch_bytes(int64_t n, int BM, int BN);
PruneOut prune_outputs(void *scratch, int64_t n, int BM, int BN);   // the launcher's output pointers
cudaError_t launch_prune_bounds(const void *Qb, int64_t n, int d, int metric, int BM, int BN, int window,
                                const float *st_key, int EG, int KCP, void *scratch, PruneOut *out,
                                cudaStream_t st);
cudaError_t launch_knn_tc_window(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh,
                                 int window, float *st_key, int32_t *st_id, unsigned int *status, cudaStream_t st);
cudaError_t launch_knn_tc_list(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh, int window,
                               const float *st_key, const int32_t *st_id, const int32_t *tiles,
                               const int64_t *tile_off, const int32_t *order, const int32_t *overflow,
                               int32_t *cand, int *counter,
                               unsigned int *status, cudaStream_t st);
// SM clock cycles each bounded wait of the tensor-core kernels may take
// before the kernel records RSC_ERR_TIMEOUT (process-wide, see
// rsc_set_wait_budget).
long long tc_wait_budget();
int knn_tc_bm();   // query rows per tensor-core work item
int knn_tc_bn();   // database rows per tensor-core tile

// ---- knn_tc_batched.cu ---------------------------------------------------------
// Batched search: one launch over (query tile of a sample) x (database sample)
// items, parts (2 or 4) threads per query row.  Within lists:
// [parts, N, kBatchedList] (re-ranked by launch_rerank with parts splits);
// cross lists: [N, S, parts * kBatchedShort] (re-ranked by launch_rerank_cross).
constexpr int kBatchedList = 16;      // within-sample ids per (row, part); k_within <= 16
constexpr int kBatchedShort = 4;      // cross-sample ids per (row, sample, part); k_cross <= 4
constexpr int kBatchedParts = 4;
// Host-built work tables (see knn_tc_batched.cu for the byte layout).
struct BatchedTables {
    int64_t *tile_row, *tile_end, *samp_off, *dtile_start, *dtile_end;
    int32_t *tile_samp, *samp_order, *counter, *dtile_off;
};
BatchedTables batched_tables(void *base, int64_t T, int S, int64_t DT);
size_t batched_tables_bytes(int64_t T, int S, int64_t DT);
int64_t batched_query_tiles(const int64_t *offsets_host, int S);
int64_t batched_db_tiles(const int64_t *offsets_host, int S);
void batched_fill_tables(const int64_t *offsets_host, int S, void *host_buf);
cudaError_t launch_knn_tc_batched(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                  int64_t DT, int parts, int stages, const void *tables_dev, int32_t *cand_w, int32_t *cand_x,
                                  unsigned int *status, cudaStream_t st);
// Pruned batched search on rows in sample-preserving locality order: a window
// pass around win[t * T + qt] saving keys (st_w [parts, N, kBatchedList],
// st_x [N, S, parts, kBatchedShort]) and ids (cand_w, cand_x), then a list
// pass over the kept tiles (tile_off over items t * T + qt).
cudaError_t launch_knn_tc_batched_window(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                         int64_t DT, int parts, int stages, const void *tables_dev, const int32_t *win, int window,
                                         float *st_w, int32_t *cand_w, float *st_x, int32_t *cand_x,
                                         unsigned int *status, cudaStream_t st);
cudaError_t launch_knn_tc_batched_list(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                       int64_t DT, int parts, int stages, const void *tables_dev, const int32_t *win, int window,
                                       const float *st_w, int32_t *cand_w, const float *st_x, int32_t *cand_x,
                                       const int32_t *tiles, const int64_t *tile_off, const int32_t *overflow,
                                       unsigned int *status, cudaStream_t st);
// perm (nullable): query and candidate positions map to original rows; R by
// position when r_by_pos.  Output rows by original row.
cudaError_t launch_rerank_cross(const float *R, int64_t rs, int64_t N, int d, int metric, const void *tables_dev,
                                int S, int T, int64_t DT, int parts, const int32_t *cand_x, const int32_t *perm,
                                bool r_by_pos, const int32_t *idx_w, const float *dist_w, int k_within, int k_cross,
                                int32_t *idx_x, float *dist_x, cudaStream_t st);
// Bounds of the pruned batched search (prune.cu): tile spheres, the nearest
// database tile of every sample for every query tile (win), tau per item from
// the window pass's saved keys, kept-tile lists per item.
struct BatchedPruneOut {
    int32_t *win;        // [S * T]
    int64_t *tile_off;   // [S * T + 1]
    int32_t *tiles;      // [cap]
    int32_t *overflow;   // [1]
};
size_t batched_prune_scratch_bytes(int64_t N, int64_t T, int S, int64_t DT);
BatchedPruneOut batched_prune_outputs(void *scratch, int64_t N, int64_t T, int S, int64_t DT);
cudaError_t launch_batched_prune_window(const void *Qb, int64_t N, int d, int metric, const void *tables_dev, int64_t T,
                                        int S, int64_t DT, void *scratch, cudaStream_t st);
cudaError_t launch_batched_prune_bounds(int64_t N, int d, int metric, const void *tables_dev, int64_t T, int S,
                                        int64_t DT, int window, int parts, const float *st_w, const float *st_x,
                                        void *scratch, cudaStream_t st);

// ---- autotune.cu --------------------------------------------------------------
// Tuned-choice table consulted when options are automatic (all zero).
struct TunedChoice {
    int db_splits, candidates, tc_parts;
    int stages = 0;   // database-tile pipeline stages (0: as many as fit)
};
bool tuned_lookup(int kind, int precision, int metric, int d, int k, int kx, int64_t n, TunedChoice *out);
void tuned_store(int kind, int precision, int metric, int d, int k, int kx, int64_t n, const TunedChoice &c);

// ---- rerank.cu ------------------------------------------------------------
// Exact re-rank: every candidate of query q (splits * KC ids, split s at
// cand[(s * n + q) * KC]) is re-scored by direct difference in FP32 over the
// rows R (row stride rs: the caller's X for Euclidean, the normalised Y for
// cosine, whose column d is the zero-row flag), sorted by (distance, id) and
// the first k written to idx/dist (Euclidean sqrt, cosine d^2 / 2 with the
// zero-row convention).  splits * KC <= 1024.
// perm (nullable): candidate lists are indexed by sorted position i, whose
// original row is perm[i]; ids in the lists are sorted positions too.  The
// output is always by original row and holds original ids.  r_by_pos: R holds
// the rows in sorted order (R row i = original row perm[i]), so the gathers of
// neighbouring queries' candidates stay close in memory.
cudaError_t launch_rerank(const float *R, int64_t rs, int64_t n, int d, int metric,
                          const int32_t *cand, int KC, int splits, int k, const int32_t *perm, bool r_by_pos,
                          int32_t *idx, float *dist, cudaStream_t st);
// dst row i <- src row perm[i] (width floats per row).
cudaError_t launch_gather_rows(const float *src, int64_t src_stride, int64_t n, int width, const int32_t *perm,
                               float *dst, int64_t dst_stride, cudaStream_t st);

// ---- connectivities.cu -------------------------------------------------------
// Shape of the connectivities passes for k: G lanes per row (16 or 32), E own
// entries per lane, KP = row stride of the sorted own entries, B = bucket
// slots per row (transposed entries that are merged in registers), MW = words
// of the per-row overflow bit mask, smooth_rows = rows per smooth-pass block.
struct ConnShape {
    int G, E, KP, B, MW, smooth_rows;
};
ConnShape conn_shape(int k);
struct ConnWork {
    unsigned int *status;
    float2 *rs;          // [n] (rho, sigma)
    float *part_sum;     // [conn_sum_blocks] distance sums of the smooth blocks
    int32_t *rho0_rows;  // [n] rows without a non-zero distance
    int32_t *ocol;       // [n, KP] own entries with a non-zero weight, by column (INT32_MAX pads)
    float *og;           // [n, KP] their values (the union value after the match pass)
    int32_t *own_cnt;    // [n]
    int2 *bucket;        // [n, B] pushed entries (source row, weight bits)
    uint32_t *ovf;       // [n, MW] pushes that found their target's bucket full
    int32_t *in_kept;    // [n] bucket entries kept by the match pass
    int64_t *local;      // [n] row offset inside its scan tile
    int64_t *scan_part;  // [scan blocks]
    int32_t *in_cnt;     // [n]   zeroed by the launcher: pushes per row
    int32_t *cursor;     // [n]   zeroed by the launcher
    int32_t *extra;      // [n]   zeroed by the launcher: flagged entries per row
    int32_t *rho0_count; // [1]   zeroed by the launcher
    int32_t *mid_count;  // [1]   zeroed by the launcher
    int32_t *long_count; // [1]   zeroed by the launcher
    int32_t *mid_rows;   // [n]
    int32_t *long_rows;  // [n]
};
size_t conn_scan_blocks(int64_t n);
size_t conn_sum_blocks(int64_t n, int k);
// Passes smooth, match and scan: rho/sigma (rho_out/sigma_out nullable),
// union values, buckets, tile offsets and indptr[n] = nnz.
cudaError_t launch_conn_count(const int32_t *idx, const float *dist, int64_t n, int k, int64_t *indptr,
                              float *rho_out, float *sigma_out, const ConnWork &w, cudaStream_t st);
// indptr[0 .. n) from the count passes (when the CSR is not filled).
cudaError_t launch_conn_indptr(int64_t n, int64_t *indptr, const ConnWork &w, cudaStream_t st);
// Passes emit and sort: indptr[0 .. n), indices and data.
cudaError_t launch_conn_fill(const int32_t *idx, const float *dist, int64_t n, int k, int64_t *indptr,
                             int32_t *indices, float *data, int64_t cap, const ConnWork &w, cudaStream_t st);

// ---- umap.cu --------------------------------------------------------------
// UMAP layout epochs (rsc_umap_layout).  Positions live in rows of
// umap_row_floats(dim) floats inside the workspace.
struct UmapParams {
    float a, b, gamma, lr;
    int neg_rate, n_epochs;
    uint64_t seed;
};
int umap_row_floats(int dim);
// *wmax_bits = largest positive weight; f[e] = data[e] / that weight;
// rowoff[e] = (row of e) mod 32.
cudaError_t launch_umap_prepare(const int64_t *indptr, const float *data, int64_t n, int64_t nnz,
                                unsigned int *wmax_bits, float *f, uint8_t *rowoff, cudaStream_t st);
// Epochs first .. last on `embedding` [n, dim] through buffers buf0/buf1.
cudaError_t launch_umap_epochs(const int64_t *indptr, const int32_t *indices, const float *f, const uint8_t *rowoff,
                               int64_t n, int64_t nnz, int dim, float *embedding, float *buf0, float *buf1, int first,
                               int last, UmapParams p, unsigned int *status, cudaStream_t st);

}  // namespace rsc
