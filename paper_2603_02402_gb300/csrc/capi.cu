// C ABI entry points (include/rsc.h): argument checks, workspace layout and
// launch sequences.  Everything numeric happens in the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

rsc_status fail(rsc_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

static std::atomic<long long> g_wait_budget{0};

long long tc_wait_budget() {
    const long long b = g_wait_budget.load(std::memory_order_relaxed);
    return b > 0 ? b : 2000000000LL;   // default: about 1 s of SM clocks
}

// ------------------------------------------------------------------ kNN plan

namespace {

constexpr int kSupportedKC[] = {16, 32, 64};

struct KnnPlan {
    int precision = RSC_FP32;
    int d = 0, metric = 0;
    int DP = 0;         // padded FP32 row length
    int KC = 0;         // ids per candidate list
    int parts = 1;      // candidate lists per query per split
    int splits = 1;     // database splits
    int64_t split_len = 0;
    bool order = false; // locality ordering before the tensor-core search
    bool prune = false; // window pass + tile bounds + list pass instead of one full scan
    int stages = 0;     // tensor-core pipeline stages (0: as many as fit)
};

struct KnnLayout {
    unsigned int *status;
    float *Y;
    float *ny;
    float *prep_scratch;
    void *Qb, *Db;       // BF16 or FP8 operands (tensor-core path only)
    unsigned int *amax;  // largest |y| (FP8 scale), FP8 only
    int32_t *cand;
    int32_t *perm;       // locality order (sorted position -> row), when planned
    void *order_scratch;
    float *Rp;           // re-rank rows in sorted order, when planned
    float *st_key;       // saved lists of the pruned search [n, parts, KC]
    int32_t *st_id;
    void *prune_scratch;
};

rsc_status plan_knn(int64_t n, int32_t d, int32_t k, int32_t metric, const rsc_knn_opts *o,
                    KnnPlan *p) {
    rsc_knn_opts def = {};
    if (!o) o = &def;
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "n=%lld out of [1, 2^31)", (long long)n);
    if (metric != RSC_EUCLIDEAN && metric != RSC_COSINE) return fail(RSC_ERR_INVALID_ARG, "unknown metric %d", metric);
    const int dmax = (metric == RSC_COSINE) ? 63 : 64;
    if (d < 1 || d > dmax) return fail(RSC_ERR_INVALID_ARG, "d=%d out of [1, %d]", d, dmax);
    if (k < 1 || k > 64 || k > n) return fail(RSC_ERR_INVALID_ARG, "k=%d out of [1, min(n, 64)]", k);
    if (o->precision != RSC_FP32 && o->precision != RSC_BF16 && o->precision != RSC_FP8)
        return fail(RSC_ERR_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->candidates < 0 || o->db_splits < 0) return fail(RSC_ERR_INVALID_ARG, "negative option");
    if (o->tc_parts != 0 && o->tc_parts != 2 && o->tc_parts != 4)
        return fail(RSC_ERR_INVALID_ARG, "tc_parts=%d (0, 2 or 4)", o->tc_parts);
    if (o->locality < 0 || o->locality > 2) return fail(RSC_ERR_INVALID_ARG, "locality=%d (0, 1 or 2)", o->locality);
    if (o->prune < 0 || o->prune > 2) return fail(RSC_ERR_INVALID_ARG, "prune=%d (0, 1 or 2)", o->prune);
    if (o->stages != 0 && (o->stages < 2 || o->stages > 6))
        return fail(RSC_ERR_INVALID_ARG, "stages=%d (0 or 2 .. 6)", o->stages);
    rsc_knn_opts tuned;
    if (o->db_splits == 0 && o->candidates == 0 && o->tc_parts == 0 && o->stages == 0) {   // automatic: tuned table first
        TunedChoice c;
        if (tuned_lookup(0, o->precision, metric, d, k, 0, n, &c)) {
            tuned = *o;
            tuned.db_splits = c.db_splits;
            tuned.candidates = c.candidates;
            tuned.tc_parts = c.tc_parts;
            tuned.stages = c.stages;
            o = &tuned;
        }
    }
    p->stages = o->stages;
    p->precision = o->precision;
    p->d = d;
    p->metric = metric;
    const bool tc = o->precision == RSC_BF16 || o->precision == RSC_FP8;   // tensor-core candidate search
    p->order = tc && (o->locality == 2 || (o->locality == 0 && n >= kOrderMinRows));
    p->DP = ((d + (metric == RSC_COSINE ? 1 : 0) + 7) / 8) * 8;
    int want = o->candidates;
    // BF16 candidates: 2k for Euclidean rows; unit-length cosine rows crowd
    // their distances together, so BF16 rounding reorders more of them: 4k
    // defaults: FP32 lists are exact up to ties (k + 8); BF16 needs 2k
    // (Euclidean) or 4k (cosine: unit-length rows crowd their distances);
    // E4M3's 3 mantissa bits need 8k
    if (want == 0)
        want = (p->precision == RSC_FP32) ? k + 8
               : (p->precision == RSC_FP8) ? 8 * k
                                           : (metric == RSC_COSINE ? 4 * k : 2 * k);
    if (want < k) return fail(RSC_ERR_INVALID_ARG, "candidates=%d smaller than k=%d", want, k);
    if (want > 64) {
        if (o->candidates != 0 && p->precision == RSC_FP32)
            return fail(RSC_ERR_INVALID_ARG, "candidates=%d above 64", want);
        if (o->candidates > 128) return fail(RSC_ERR_INVALID_ARG, "candidates=%d above 128", want);
        if (o->candidates == 0)
            want = ((metric == RSC_COSINE && p->precision == RSC_BF16) || p->precision == RSC_FP8) ? std::min(want, 128)
                                                                                                  : 64;
    }
    // candidates per row: FP32 lists of KC; tensor-core rows as parts x list
    p->KC = 0;
    p->parts = 1;
    if (tc) {
        if (!knn_tc_supported(d, metric)) return fail(RSC_ERR_UNSUPPORTED, "no tensor-core kernel for d=%d", d);
        if (p->precision == RSC_FP8 && !knn_tc_fp8_supported(d, metric))
            return fail(RSC_ERR_UNSUPPORTED, "no FP8 kernel for d=%d (d + %d <= 64)", d,
                        metric == RSC_EUCLIDEAN ? 5 : 1);
        TcShape sh = knn_tc_shape(d, metric, k, want, o->tc_parts);
        if (sh.parts == 0) return fail(RSC_ERR_UNSUPPORTED, "no tensor-core list shape for k=%d candidates=%d", k, want);
        p->parts = sh.parts;
        p->KC = sh.list;
    } else {
        for (int c : kSupportedKC)
            if (c >= want) { p->KC = c; break; }
        if (!knn_simt_supported(p->DP, p->KC))
            return fail(RSC_ERR_UNSUPPORTED, "no SIMT kernel for DP=%d KC=%d", p->DP, p->KC);
    }
    // database splits: enough CTAs to fill the GPU when there are few queries
    const int64_t qrows = tc ? 128 : 256;             // query rows per CTA work unit
    const int64_t target = 152;                       // work units wanted (persistent CTAs)
    const int64_t align = tc ? knn_tc_split_align() : 64;
    const int64_t qblocks = ceil_div(n, qrows);
    const int per_split = p->parts * p->KC;           // candidate ids per row and split
    int splits = o->db_splits;
    if (splits == 0 && !tc) {
        // one CTA per SM: the fewest splits whose waves are at least 94 % full
        // (each split adds a candidate list per row), else the fullest
        double best = -1.0;
        for (int s = 1; s <= 8; ++s) {
            const int64_t ctas = qblocks * s, waves = ceil_div(ctas, (int64_t)152);
            const double fill = (double)ctas / (double)(152 * waves);
            if (fill >= 0.94) {
                splits = s;
                break;
            }
            if (fill > best + 1e-9) {
                best = fill;
                splits = s;
            }
        }
    }
    if (splits == 0) splits = (int)std::min<int64_t>(8, std::max<int64_t>(1, ceil_div(target, qblocks)));
    while (splits > 1 && splits * per_split > 1024) --splits;
    if (splits * per_split > 1024) return fail(RSC_ERR_INVALID_ARG, "db_splits * candidates above 1024");
    p->split_len = ceil_div(ceil_div(n, splits), align) * align;
    p->splits = (int)ceil_div(n, p->split_len);
    // pruning: BF16 rows in locality order, one database split, one 64-element K block
    const bool prune_ok = p->order && p->splits == 1 && p->precision == RSC_BF16 && tc_kb(d, metric) == 1;
    if (o->prune == 2 && !prune_ok)
        return fail(RSC_ERR_UNSUPPORTED, "prune needs BF16, the locality ordering, one database split and d + 3 <= 64");
    p->prune = prune_ok && o->prune != 1;
    return RSC_OK;
}

KnnLayout carve_knn(void *ws, int64_t n, const KnnPlan &p, size_t *bytes) {
    Carve cv(ws);
    KnnLayout L;
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.Y = cv.take<float>((size_t)n * p.DP);
    L.ny = cv.take<float>((size_t)n);
    L.prep_scratch = cv.take<float>(prep_scratch_floats());
    L.Qb = L.Db = nullptr;
    L.amax = nullptr;
    if (p.precision == RSC_BF16) {
        L.Qb = cv.take<uint16_t>((size_t)n * 64 * tc_kb(p.d, p.metric));
        L.Db = cv.take<uint16_t>((size_t)n * 64 * tc_kb(p.d, p.metric));
    } else if (p.precision == RSC_FP8) {
        L.Qb = cv.take<uint8_t>((size_t)n * 64);
        L.Db = cv.take<uint8_t>((size_t)n * 64);
        L.amax = cv.take<unsigned int>(1);
    }
    L.cand = cv.take<int32_t>((size_t)p.splits * p.parts * n * p.KC);
    L.perm = nullptr;
    L.order_scratch = nullptr;
    L.Rp = nullptr;
    if (p.order) {
        L.perm = cv.take<int32_t>((size_t)n);
        L.order_scratch = cv.take<uint8_t>(order_scratch_bytes(n, p.DP));
        L.Rp = cv.take<float>((size_t)n * (p.metric == RSC_EUCLIDEAN ? ceil_div(p.d, 4) * 4 : p.DP));
    }
    L.st_key = nullptr;
    L.st_id = nullptr;
    L.prune_scratch = nullptr;
    if (p.prune) {
        L.st_key = cv.take<float>((size_t)n * p.parts * p.KC);
        L.st_id = cv.take<int32_t>((size_t)n * p.parts * p.KC);
        L.prune_scratch = cv.take<uint8_t>(prune_scratch_bytes(n, knn_tc_bm(), knn_tc_bn()));
    }
    if (bytes) *bytes = cv.used;
    return L;
}

rsc_status check_ws(void *ws, size_t have, size_t need) {
    if (!ws) return fail(RSC_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(RSC_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (have < need) return fail(RSC_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", have, need);
    return RSC_OK;
}

// ------------------------------------------------------- connectivities plan

struct ConnLayout {
    ConnWork w;
    int64_t *indptr_tmp;
    int32_t *zeroed;       // in_cnt, cursor, extra, rho0_count, mid_count, long_count (3n + 3 int32)
};

ConnLayout carve_conn(void *ws, int64_t n, int k, size_t *bytes) {
    const ConnShape s = conn_shape(k);
    Carve cv(ws);
    ConnLayout L;
    L.w.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.w.rs = cv.take<float2>((size_t)n);
    L.w.part_sum = cv.take<float>(conn_sum_blocks(n, k));
    L.w.rho0_rows = cv.take<int32_t>((size_t)n);
    L.w.ocol = cv.take<int32_t>((size_t)n * s.KP);
    L.w.og = cv.take<float>((size_t)n * s.KP);
    L.w.own_cnt = cv.take<int32_t>((size_t)n);
    L.w.bucket = cv.take<int2>((size_t)n * s.B);
    L.w.ovf = cv.take<uint32_t>((size_t)n * s.MW);
    L.w.in_kept = cv.take<int32_t>((size_t)n);
    L.w.local = cv.take<int64_t>((size_t)n);
    L.w.scan_part = cv.take<int64_t>(conn_scan_blocks(n));
    L.zeroed = cv.take<int32_t>((size_t)3 * n + 3);
    L.w.in_cnt = L.zeroed;
    L.w.cursor = L.zeroed ? L.zeroed + n : nullptr;
    L.w.extra = L.zeroed ? L.zeroed + 2 * n : nullptr;
    L.w.rho0_count = L.zeroed ? L.zeroed + 3 * n : nullptr;
    L.w.mid_count = L.zeroed ? L.zeroed + 3 * n + 1 : nullptr;
    L.w.long_count = L.zeroed ? L.zeroed + 3 * n + 2 : nullptr;
    L.w.mid_rows = cv.take<int32_t>((size_t)n);
    L.w.long_rows = cv.take<int32_t>((size_t)n);
    L.indptr_tmp = cv.take<int64_t>((size_t)n + 1);
    if (bytes) *bytes = cv.used;
    return L;
}

rsc_status check_conn_args(const int32_t *idx, const float *dist, int64_t n, int32_t k) {
    if (!idx || !dist) return fail(RSC_ERR_INVALID_ARG, "idx/dist is NULL");
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "n=%lld out of [1, 2^31)", (long long)n);
    if (k < 1 || k > 256) return fail(RSC_ERR_INVALID_ARG, "k=%d out of [1, 256]", k);
    return RSC_OK;
}

rsc_status conn_count_phase(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                            int64_t *indptr, float *rho, float *sigma, ConnLayout &L,
                            cudaStream_t st) {
    RSC_CUDA_TRY(cudaMemsetAsync(L.w.status, 0, sizeof(unsigned int), st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.zeroed, 0, sizeof(int32_t) * (3 * n + 3), st));
    RSC_CUDA_TRY(launch_conn_count(idx, dist, n, k, indptr, rho, sigma, L.w, st));
    return RSC_OK;
}

// ------------------------------------------------------------- batched plan

struct BatchedPlan {
    int64_t n = 0;
    int d = 0, S = 0, kw = 0, kx = 0, metric = 0, DP = 0;
    int parts = 4;      // threads (column parts) per query row
    int stages = 0;     // tensor-core pipeline stages (0: as many as fit)
    int64_t T = 0;      // query tiles (128 rows inside one sample)
    int64_t DT = 0;     // database tiles (256 rows inside one sample)
    bool order = false; // rows in cluster order inside each sample
    bool prune = false; // window pass + tile bounds + list pass
};

struct BatchedLayout {
    unsigned int *status;
    float *Y, *ny, *prep_scratch;
    void *Qb, *Db;
    void *tables;
    int32_t *cand_w, *cand_x;
    int32_t *perm;             // ordering
    void *order_scratch;
    float *Rp;                 // re-rank rows in sorted order
    float *st_w, *st_x;        // saved keys of the pruned search
    void *prune_scratch;
};

rsc_status plan_batched(int64_t n, int32_t d, const int64_t *off, int32_t S, int32_t kw, int32_t kx,
                        int32_t metric, const rsc_knn_opts *o, BatchedPlan *p) {
    rsc_knn_opts def = {};
    if (!o) o = &def;
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "n=%lld out of [1, 2^31)", (long long)n);
    if (metric != RSC_EUCLIDEAN && metric != RSC_COSINE) return fail(RSC_ERR_INVALID_ARG, "unknown metric %d", metric);
    if (d < 1 || d + (metric == RSC_EUCLIDEAN ? 3 : 1) > 64)
        return fail(d < 1 ? RSC_ERR_INVALID_ARG : RSC_ERR_UNSUPPORTED, "d=%d not supported by the batched search", d);
    if (!off || S < 1) return fail(RSC_ERR_INVALID_ARG, "sample_offsets / n_samples");
    if (kw < 1 || kw > kBatchedList) return fail(RSC_ERR_INVALID_ARG, "k_within=%d out of [1, %d]", kw, kBatchedList);
    if (kx < 1 || kx > kBatchedShort || kx > kw)
        return fail(RSC_ERR_INVALID_ARG, "k_cross=%d out of [1, min(%d, k_within)]", kx, kBatchedShort);
    if ((int64_t)S * kx > 1024) return fail(RSC_ERR_INVALID_ARG, "n_samples * k_cross above 1024");
    if (o->precision != RSC_BF16) return fail(RSC_ERR_UNSUPPORTED, "batched search runs BF16 candidates only");
    if (o->tc_parts != 0 && o->tc_parts != 2 && o->tc_parts != 4)
        return fail(RSC_ERR_INVALID_ARG, "tc_parts=%d (0, 2 or 4)", o->tc_parts);
    if (o->stages != 0 && (o->stages < 2 || o->stages > 6))
        return fail(RSC_ERR_INVALID_ARG, "stages=%d (0 or 2 .. 6)", o->stages);
    p->parts = o->tc_parts;
    p->stages = o->stages;
    if (p->parts == 0) {
        TunedChoice c;
        const bool hit = tuned_lookup(1, o->precision, metric, d, kw, kx, n, &c);
        p->parts = hit ? c.tc_parts : 4;
        if (hit && o->stages == 0) p->stages = c.stages;
    }
    if (off[0] != 0 || off[S] != n) return fail(RSC_ERR_INVALID_ARG, "sample_offsets must run from 0 to n");
    for (int s = 0; s < S; ++s)
        if (off[s + 1] - off[s] < kw) return fail(RSC_ERR_INVALID_ARG, "sample %d has fewer than k_within cells", s);
    p->n = n;
    p->d = d;
    p->S = S;
    p->kw = kw;
    p->kx = kx;
    p->metric = metric;
    p->DP = ((d + (metric == RSC_COSINE ? 1 : 0) + 7) / 8) * 8;
    p->T = batched_query_tiles(off, S);
    p->DT = batched_db_tiles(off, S);
    if (p->T * S >= (int64_t(1) << 31)) return fail(RSC_ERR_UNSUPPORTED, "too many (tile, sample) work items");
    if (o->locality < 0 || o->locality > 2) return fail(RSC_ERR_INVALID_ARG, "locality=%d (0, 1 or 2)", o->locality);
    if (o->prune < 0 || o->prune > 2) return fail(RSC_ERR_INVALID_ARG, "prune=%d (0, 1 or 2)", o->prune);
    const bool order_ok = S <= kOrderMaxLeaves;
    if (o->locality == 2 && !order_ok) return fail(RSC_ERR_UNSUPPORTED, "locality ordering supports %d samples", kOrderMaxLeaves);
    p->order = order_ok && (o->locality == 2 || (o->locality == 0 && n >= kOrderMinRows));
    if (o->prune == 2 && !p->order) return fail(RSC_ERR_UNSUPPORTED, "prune needs the locality ordering");
    p->prune = p->order && o->prune != 1;
    return RSC_OK;
}

BatchedLayout carve_batched(void *ws, const BatchedPlan &p, size_t *bytes) {
    Carve cv(ws);
    BatchedLayout L;
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.Y = cv.take<float>((size_t)p.n * p.DP);
    L.ny = cv.take<float>((size_t)p.n);
    L.prep_scratch = cv.take<float>(prep_scratch_floats());
    L.Qb = cv.take<uint16_t>((size_t)p.n * 64);
    L.Db = cv.take<uint16_t>((size_t)p.n * 64);
    L.tables = cv.take<uint8_t>(batched_tables_bytes(p.T, p.S, p.DT));
    // sized for the widest part count, so a tuned choice always fits
    L.cand_w = cv.take<int32_t>((size_t)kBatchedParts * p.n * kBatchedList);
    L.cand_x = cv.take<int32_t>((size_t)p.n * p.S * kBatchedParts * kBatchedShort);
    L.perm = nullptr;
    L.order_scratch = nullptr;
    L.Rp = nullptr;
    L.st_w = L.st_x = nullptr;
    L.prune_scratch = nullptr;
    if (p.order) {
        L.perm = cv.take<int32_t>((size_t)p.n);
        L.order_scratch = cv.take<uint8_t>(order_scratch_bytes(p.n, p.DP, p.S));
        L.Rp = cv.take<float>((size_t)p.n * (p.metric == RSC_EUCLIDEAN ? ceil_div(p.d, 4) * 4 : p.DP));
    }
    if (p.prune) {
        L.st_w = cv.take<float>((size_t)kBatchedParts * p.n * kBatchedList);
        L.st_x = cv.take<float>((size_t)p.n * p.S * kBatchedParts * kBatchedShort);
        L.prune_scratch = cv.take<uint8_t>(batched_prune_scratch_bytes(p.n, p.T, p.S, p.DT));
    }
    if (bytes) *bytes = cv.used;
    return L;
}

rsc_status enqueue_batched(const float *X, const BatchedPlan &p, const BatchedLayout &L, const void *tables_host,
                           int32_t *iw, float *dw, int32_t *ix, float *dx, cudaStream_t st) {
    const int64_t n = p.n;
    const int d = p.d, metric = p.metric;
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));
    RSC_CUDA_TRY(cudaMemcpyAsync(L.tables, tables_host, batched_tables_bytes(p.T, p.S, p.DT), cudaMemcpyHostToDevice,
                                 st));
    RSC_CUDA_TRY(launch_prep_fp32(X, n, d, p.DP, metric, L.Y, L.ny, L.prep_scratch, st));
    const BatchedTables tb = batched_tables(L.tables, p.T, p.S, p.DT);
    if (p.order)   // cluster order inside each sample (the samples keep their row ranges)
        RSC_CUDA_TRY(launch_locality_order(L.Y, n, p.DP, kOrderIters, L.perm, L.order_scratch, st, tb.samp_off, p.S));
    RSC_CUDA_TRY(launch_prep_bf16(L.Y, n, d, p.DP, metric, L.perm, L.Qb, L.Db, st));
    if (p.prune) {
        const BatchedPruneOut po = batched_prune_outputs(L.prune_scratch, n, p.T, p.S, p.DT);
        RSC_CUDA_TRY(launch_batched_prune_window(L.Qb, n, d, metric, L.tables, p.T, p.S, p.DT, L.prune_scratch, st));
        RSC_CUDA_TRY(launch_knn_tc_batched_window(L.Qb, L.Db, n, d, metric, p.S, (int)p.T, p.DT, p.parts, p.stages, L.tables,
                                                  po.win, kOrderWindow, L.st_w, L.cand_w, L.st_x, L.cand_x, L.status,
                                                  st));
        RSC_CUDA_TRY(launch_batched_prune_bounds(n, d, metric, L.tables, p.T, p.S, p.DT, kOrderWindow, p.parts, L.st_w,
                                                 L.st_x, L.prune_scratch, st));
        RSC_CUDA_TRY(launch_knn_tc_batched_list(L.Qb, L.Db, n, d, metric, p.S, (int)p.T, p.DT, p.parts, p.stages, L.tables,
                                                po.win, kOrderWindow, L.st_w, L.cand_w, L.st_x, L.cand_x, po.tiles,
                                                po.tile_off, po.overflow, L.status, st));
    } else {
        RSC_CUDA_TRY(launch_knn_tc_batched(L.Qb, L.Db, n, d, metric, p.S, (int)p.T, p.DT, p.parts, p.stages, L.tables,
                                           L.cand_w, L.cand_x, L.status, st));
    }
    const float *R = (metric == RSC_EUCLIDEAN) ? X : L.Y;
    int64_t rs = (metric == RSC_EUCLIDEAN) ? d : p.DP;
    if (p.order) {   // rows in search order, 16-byte aligned
        const int64_t rsr = (metric == RSC_EUCLIDEAN) ? ceil_div(d, 4) * 4 : p.DP;
        RSC_CUDA_TRY(launch_gather_rows(R, rs, n, (int)rs, L.perm, L.Rp, rsr, st));
        R = L.Rp;
        rs = rsr;
    }
    RSC_CUDA_TRY(launch_rerank(R, rs, n, d, metric, L.cand_w, kBatchedList, p.parts, p.kw, L.perm, p.order, iw, dw,
                               st));
    RSC_CUDA_TRY(launch_rerank_cross(R, rs, n, d, metric, L.tables, p.S, (int)p.T, p.DT, p.parts, L.cand_x, L.perm,
                                     p.order, iw, dw, p.kw, p.kx, ix, dx, st));
    return RSC_OK;
}

// CUDA graphs of the batched launch sequence, one per argument set.  The
// host copy of the work tables lives in pinned memory owned by the entry so
// that every replay re-uploads them (the workspace may have been reused).
struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    void *tables_pinned = nullptr;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxGraphs = 8;

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" {

const char *rsc_version(void) { return "rsc-gb300 0.1 (sm_103a)"; }

const char *rsc_last_error(void) { return g_err; }

rsc_status rsc_set_wait_budget(int64_t clocks) {
    if (clocks < 0) return fail(RSC_ERR_INVALID_ARG, "negative wait budget");
    g_wait_budget.store((long long)clocks, std::memory_order_relaxed);
    return RSC_OK;
}

rsc_status rsc_workspace_status(void *workspace, void *stream) {
    if (!workspace) return fail(RSC_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int word = 0;
    RSC_CUDA_TRY(cudaMemcpyAsync(&word, workspace, sizeof(word), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    RSC_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(word), st));
    if (word != 0) return fail((rsc_status)word, "a kernel recorded status %u", word);
    return RSC_OK;
}

rsc_status rsc_knn_workspace_size(int64_t n, int32_t d, int32_t k, int32_t metric,
                                  const rsc_knn_opts *opts, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    KnnPlan p;
    rsc_status s = plan_knn(n, d, k, metric, opts, &p);
    if (s != RSC_OK) return s;
    carve_knn(nullptr, n, p, bytes);
    return RSC_OK;
}

rsc_status rsc_knn(const float *X, int64_t n, int32_t d, int32_t k, int32_t metric, int32_t *idx,
                   float *dist, const rsc_knn_opts *opts, void *workspace, size_t workspace_bytes) {
    RSC_TRACE("rsc_knn");
    if (!X || !idx || !dist) return fail(RSC_ERR_INVALID_ARG, "X/idx/dist is NULL");
    KnnPlan p;
    rsc_status s = plan_knn(n, d, k, metric, opts, &p);
    if (s != RSC_OK) return s;
    size_t need = 0;
    carve_knn(nullptr, n, p, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    KnnLayout L = carve_knn(workspace, n, p, nullptr);
    cudaStream_t st = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
    cudaEvent_t *ev = opts ? static_cast<cudaEvent_t *>(opts->phase_events) : nullptr;
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));
    if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[0], st));
    RSC_CUDA_TRY(launch_prep_fp32(X, n, d, p.DP, metric, L.Y, L.ny, L.prep_scratch, st));
    if (p.precision == RSC_BF16) {
        if (p.order) RSC_CUDA_TRY(launch_locality_order(L.Y, n, p.DP, kOrderIters, L.perm, L.order_scratch, st));
        RSC_CUDA_TRY(launch_prep_bf16(L.Y, n, d, p.DP, metric, L.perm, L.Qb, L.Db, st));
        if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[1], st));
        const TcShape sh{p.parts, p.KC, p.stages};
        if (p.prune) {
            RSC_CUDA_TRY(launch_knn_tc_window(L.Qb, L.Db, n, d, metric, sh, kOrderWindow, L.st_key, L.st_id, L.status,
                                              st));
            PruneOut po;
            RSC_CUDA_TRY(launch_prune_bounds(L.Qb, n, d, metric, knn_tc_bm(), knn_tc_bn(), kOrderWindow, L.st_key,
                                             p.parts, p.KC, L.prune_scratch, &po, st));
            RSC_CUDA_TRY(launch_knn_tc_list(L.Qb, L.Db, n, d, metric, sh, kOrderWindow, L.st_key, L.st_id, po.tiles,
                                            po.tile_off, po.order, po.overflow, L.cand, po.counter, L.status, st));
        } else {
            RSC_CUDA_TRY(launch_knn_tc(L.Qb, L.Db, n, d, metric, sh, p.splits, p.split_len,
                                       p.order ? kOrderWindow : 0, L.cand, L.status, st));
        }
    } else if (p.precision == RSC_FP8) {
        if (p.order) RSC_CUDA_TRY(launch_locality_order(L.Y, n, p.DP, kOrderIters, L.perm, L.order_scratch, st));
        RSC_CUDA_TRY(launch_prep_fp8(L.Y, n, d, p.DP, metric, L.perm, L.Qb, L.Db, L.amax, st));
        if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[1], st));
        RSC_CUDA_TRY(launch_knn_tc_fp8(L.Qb, L.Db, n, d, metric, TcShape{p.parts, p.KC, p.stages}, p.splits, p.split_len,
                                       p.order ? kOrderWindow : 0, L.cand, L.status, st));
    } else {
        if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[1], st));
        RSC_CUDA_TRY(launch_knn_simt(L.Y, L.ny, n, p.DP, d + (metric == RSC_COSINE ? 1 : 0), p.KC, p.splits,
                                     p.split_len, L.cand, st));
    }
    if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[2], st));
    // exact re-rank reads the caller's rows (Euclidean) or the normalised rows (cosine)
    const float *R = (metric == RSC_EUCLIDEAN) ? X : L.Y;
    const int64_t rs = (metric == RSC_EUCLIDEAN) ? d : p.DP;
    int64_t rsr = rs;
    if (p.order) {   // rows in search order, 16-byte aligned: neighbouring queries share cache lines
        rsr = (metric == RSC_EUCLIDEAN) ? ceil_div(d, 4) * 4 : p.DP;
        RSC_CUDA_TRY(launch_gather_rows(R, rs, n, (int)rs, L.perm, L.Rp, rsr, st));
        R = L.Rp;
    }
    RSC_CUDA_TRY(launch_rerank(R, rsr, n, d, metric, L.cand, p.KC, p.splits * p.parts, k, L.perm, p.order, idx, dist,
                               st));
    if (ev) RSC_CUDA_TRY(cudaEventRecord(ev[3], st));
    return RSC_OK;
}

rsc_status rsc_knn_scan_stats(int64_t n, int32_t d, int32_t k, int32_t metric, const rsc_knn_opts *opts,
                              void *workspace, size_t workspace_bytes, int64_t *pairs_scanned,
                              int64_t *pairs_total) {
    if (!pairs_scanned || !pairs_total) return fail(RSC_ERR_INVALID_ARG, "NULL output");
    KnnPlan p;
    rsc_status s = plan_knn(n, d, k, metric, opts, &p);
    if (s != RSC_OK) return s;
    size_t need = 0;
    carve_knn(nullptr, n, p, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    const int BM = knn_tc_bm(), BN = p.precision != RSC_FP32 ? knn_tc_bn() : BM;
    const int64_t qt = ceil_div(n, BM), dt = ceil_div(n, BN);
    *pairs_total = qt * dt;
    *pairs_scanned = *pairs_total;
    if (!p.prune) return RSC_OK;
    KnnLayout L = carve_knn(workspace, n, p, nullptr);
    const PruneOut po = prune_outputs(L.prune_scratch, n, BM, BN);
    cudaStream_t st = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
    int64_t kept = 0;
    int32_t overflow = 0;
    RSC_CUDA_TRY(cudaMemcpyAsync(&kept, po.tile_off + qt, sizeof(kept), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaMemcpyAsync(&overflow, po.overflow, sizeof(overflow), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    if (overflow) return RSC_OK;   // the list pass scanned every tile
    int64_t window = 0;
    for (int64_t q = 0; q < qt; ++q) {
        const int64_t tq = q * BM / BN;
        window += std::min<int64_t>(dt, tq + kOrderWindow + 1) - std::max<int64_t>(0, tq - kOrderWindow);
    }
    *pairs_scanned = window + kept;
    return RSC_OK;
}

rsc_status rsc_knn_batched_workspace_size(int64_t n, int32_t d, const int64_t *sample_offsets,
                                          int32_t n_samples, int32_t k_within, int32_t k_cross,
                                          int32_t metric, const rsc_knn_opts *opts, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    BatchedPlan p;
    rsc_status s = plan_batched(n, d, sample_offsets, n_samples, k_within, k_cross, metric, opts, &p);
    if (s != RSC_OK) return s;
    carve_batched(nullptr, p, bytes);
    return RSC_OK;
}

rsc_status rsc_knn_batched(const float *X, int64_t n, int32_t d, const int64_t *sample_offsets,
                           int32_t n_samples, int32_t k_within, int32_t k_cross, int32_t metric,
                           int32_t *idx_within, float *dist_within, int32_t *idx_cross,
                           float *dist_cross, const rsc_knn_opts *opts, void *workspace,
                           size_t workspace_bytes) {
    RSC_TRACE("rsc_knn_batched");
    if (!X || !idx_within || !dist_within || !idx_cross || !dist_cross)
        return fail(RSC_ERR_INVALID_ARG, "NULL array argument");
    BatchedPlan p;
    rsc_status s = plan_batched(n, d, sample_offsets, n_samples, k_within, k_cross, metric, opts, &p);
    if (s != RSC_OK) return s;
    size_t need = 0;
    carve_batched(nullptr, p, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    BatchedLayout L = carve_batched(workspace, p, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
    const size_t tb = batched_tables_bytes(p.T, p.S, p.DT);
    if (st == nullptr) {   // legacy default stream cannot be captured: launch directly
        std::vector<uint8_t> host(tb);
        batched_fill_tables(sample_offsets, n_samples, host.data());
        s = enqueue_batched(X, p, L, host.data(), idx_within, dist_within, idx_cross, dist_cross, st);
        if (s == RSC_OK) RSC_CUDA_TRY(cudaStreamSynchronize(st));   // host table buffer goes out of scope
        return s;
    }
    std::vector<uint64_t> key = {(uint64_t)X, (uint64_t)n, (uint64_t)d, (uint64_t)n_samples, (uint64_t)k_within,
                                 (uint64_t)k_cross, (uint64_t)metric, (uint64_t)idx_within, (uint64_t)dist_within,
                                 (uint64_t)idx_cross, (uint64_t)dist_cross, (uint64_t)workspace,
                                 (uint64_t)p.parts, (uint64_t)p.order, (uint64_t)p.prune, (uint64_t)p.stages};
    for (int i = 0; i <= n_samples; ++i) key.push_back((uint64_t)sample_offsets[i]);
    int dev = 0;
    RSC_CUDA_TRY(cudaGetDevice(&dev));
    key.push_back((uint64_t)dev);
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto &g : g_graphs) {
        if (g.key == key) {
            RSC_CUDA_TRY(cudaGraphLaunch(g.exec, st));
            return RSC_OK;
        }
    }
    GraphEntry e;
    e.key = key;
    RSC_CUDA_TRY(cudaHostAlloc(&e.tables_pinned, tb, cudaHostAllocDefault));
    batched_fill_tables(sample_offsets, n_samples, e.tables_pinned);
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {   // e.g. the caller is capturing this stream already
        cudaGetLastError();
        s = enqueue_batched(X, p, L, e.tables_pinned, idx_within, dist_within, idx_cross, dist_cross, st);
        cudaStreamSynchronize(st);
        cudaFreeHost(e.tables_pinned);
        return s;
    }
    s = enqueue_batched(X, p, L, e.tables_pinned, idx_within, dist_within, idx_cross, dist_cross, st);
    ce = cudaStreamEndCapture(st, &graph);
    if (s != RSC_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaFreeHost(e.tables_pinned);
        return s != RSC_OK ? s : fail(RSC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        cudaFreeHost(e.tables_pinned);
        return fail(RSC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    if (g_graphs.size() >= kMaxGraphs) {   // evict the oldest entry
        cudaStreamSynchronize(st);
        cudaGraphExecDestroy(g_graphs.front().exec);
        cudaFreeHost(g_graphs.front().tables_pinned);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(e);
    RSC_CUDA_TRY(cudaGraphLaunch(e.exec, st));
    return RSC_OK;
}

rsc_status rsc_knn_batched_scan_stats(int64_t n, int32_t d, const int64_t *sample_offsets, int32_t n_samples,
                                      int32_t k_within, int32_t k_cross, int32_t metric,
                                      const rsc_knn_opts *opts, void *workspace, size_t workspace_bytes,
                                      int64_t *pairs_scanned, int64_t *pairs_total) {
    if (!pairs_scanned || !pairs_total) return fail(RSC_ERR_INVALID_ARG, "NULL output");
    BatchedPlan p;
    rsc_status s = plan_batched(n, d, sample_offsets, n_samples, k_within, k_cross, metric, opts, &p);
    if (s != RSC_OK) return s;
    size_t need = 0;
    carve_batched(nullptr, p, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    *pairs_total = p.T * p.DT;   // every query tile against every sample's database tiles
    *pairs_scanned = *pairs_total;
    if (!p.prune) return RSC_OK;
    BatchedLayout L = carve_batched(workspace, p, nullptr);
    const BatchedPruneOut po = batched_prune_outputs(L.prune_scratch, n, p.T, p.S, p.DT);
    cudaStream_t st = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
    const int64_t items = p.T * p.S;
    int64_t kept = 0;
    int32_t overflow = 0;
    std::vector<int32_t> win((size_t)items);
    RSC_CUDA_TRY(cudaMemcpyAsync(&kept, po.tile_off + items, sizeof(kept), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaMemcpyAsync(&overflow, po.overflow, sizeof(overflow), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaMemcpyAsync(win.data(), po.win, sizeof(int32_t) * (size_t)items, cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    if (overflow) return RSC_OK;   // the list pass scanned every tile
    // window tiles of item t * T + qt: sample t's tiles around win[item], +- kOrderWindow
    const int BN = knn_tc_bn();
    int64_t window = 0;
    for (int t = 0; t < n_samples; ++t) {
        const int64_t Tt = ceil_div(sample_offsets[t + 1] - sample_offsets[t], BN);
        for (int64_t qt = 0; qt < p.T; ++qt) {
            const int64_t w = win[(size_t)(t * p.T + qt)];
            window += std::min<int64_t>(Tt, w + kOrderWindow + 1) - std::max<int64_t>(0, w - kOrderWindow);
        }
    }
    *pairs_scanned = window + kept;
    return RSC_OK;
}

int64_t rsc_connectivities_max_nnz(int64_t n, int32_t k) {
    if (n < 1 || k < 1) return 0;
    return 2 * n * (int64_t)(k - 1);
}

rsc_status rsc_connectivities_workspace_size(int64_t n, int32_t k, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    if (n < 1 || k < 1 || k > 256) return fail(RSC_ERR_INVALID_ARG, "bad n/k");
    carve_conn(nullptr, n, k, bytes);
    return RSC_OK;
}

rsc_status rsc_connectivities(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                              int64_t *indptr, int32_t *indices, float *data, int64_t nnz_capacity,
                              float *rho, float *sigma, void *workspace, size_t workspace_bytes,
                              void *stream) {
    RSC_TRACE("rsc_connectivities");
    rsc_status s = check_conn_args(idx, dist, n, k);
    if (s != RSC_OK) return s;
    if (!indptr) return fail(RSC_ERR_INVALID_ARG, "indptr is NULL");
    if (nnz_capacity < 0) return fail(RSC_ERR_INVALID_ARG, "negative capacity");
    if (nnz_capacity > 0 && (!indices || !data)) return fail(RSC_ERR_INVALID_ARG, "indices/data is NULL");
    size_t need = 0;
    carve_conn(nullptr, n, k, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    ConnLayout L = carve_conn(workspace, n, k, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = conn_count_phase(idx, dist, n, k, indptr, rho, sigma, L, st)) != RSC_OK) return s;
    if (nnz_capacity < rsc_connectivities_max_nnz(n, k)) {
        int64_t nnz = 0;
        RSC_CUDA_TRY(cudaMemcpyAsync(&nnz, indptr + n, sizeof(nnz), cudaMemcpyDeviceToHost, st));
        RSC_CUDA_TRY(cudaStreamSynchronize(st));
        if (nnz > nnz_capacity) {
            RSC_CUDA_TRY(launch_conn_indptr(n, indptr, L.w, st));
            return fail(RSC_ERR_CAPACITY, "nnz=%lld exceeds capacity %lld", (long long)nnz, (long long)nnz_capacity);
        }
    }
    RSC_CUDA_TRY(launch_conn_fill(idx, dist, n, k, indptr, indices, data, nnz_capacity, L.w, st));
    return RSC_OK;
}

rsc_status rsc_connectivities_nnz(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                                  int64_t *nnz, void *workspace, size_t workspace_bytes,
                                  void *stream) {
    RSC_TRACE("rsc_connectivities_nnz");
    rsc_status s = check_conn_args(idx, dist, n, k);
    if (s != RSC_OK) return s;
    if (!nnz) return fail(RSC_ERR_INVALID_ARG, "nnz is NULL");
    size_t need = 0;
    carve_conn(nullptr, n, k, &need);
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    ConnLayout L = carve_conn(workspace, n, k, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = conn_count_phase(idx, dist, n, k, L.indptr_tmp, nullptr, nullptr, L, st)) != RSC_OK) return s;
    RSC_CUDA_TRY(cudaMemcpyAsync(nnz, L.indptr_tmp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    return RSC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- UMAP layout

namespace rsc {
namespace {

struct UmapLayout {
    unsigned int *status;
    unsigned int *wmax;
    float *f;
    uint8_t *rowoff;
    float *buf0, *buf1;
};

UmapLayout carve_umap(void *ws, int64_t n, int64_t nnz, int dim, size_t *bytes) {
    Carve cv(ws);
    UmapLayout L;
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.wmax = cv.take<unsigned int>(1);
    L.f = cv.take<float>((size_t)std::max<int64_t>(nnz, 1));
    L.rowoff = cv.take<uint8_t>((size_t)std::max<int64_t>(nnz, 1));
    L.buf0 = cv.take<float>((size_t)n * umap_row_floats(dim));
    L.buf1 = cv.take<float>((size_t)n * umap_row_floats(dim));
    if (bytes) *bytes = cv.used;
    return L;
}

// Sum of squared residuals of 1 / (1 + a x^(2b)) against the UMAP target curve.
double umap_ab_sse(const double *x, const double *y, int m, double a, double b) {
    double s = 0.0;
    for (int t = 0; t < m; ++t) {
        const double r = 1.0 / (1.0 + a * pow(x[t], 2.0 * b)) - y[t];
        s += r * r;
    }
    return s;
}

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" {

rsc_status rsc_umap_find_ab(float spread, float min_dist, float *a_out, float *b_out) {
    if (!a_out || !b_out) return fail(RSC_ERR_INVALID_ARG, "NULL output");
    if (!(spread > 0.f) || !(min_dist >= 0.f) || !std::isfinite(spread) || !std::isfinite(min_dist))
        return fail(RSC_ERR_INVALID_ARG, "spread=%g, min_dist=%g", spread, min_dist);
    constexpr int m = 300;
    double x[m], y[m];
    for (int t = 0; t < m; ++t) {
        x[t] = 3.0 * spread * t / (m - 1);
        y[t] = x[t] < min_dist ? 1.0 : exp(-(x[t] - min_dist) / spread);
    }
    // Levenberg-Marquardt on (a, b), damping on the diagonal of J^T J.
    double a = 1.0, b = 1.0, lam = 1e-3;
    double sse = umap_ab_sse(x, y, m, a, b);
    bool done = false;
    for (int it = 0; it < 1000 && !done; ++it) {
        double jtj[3] = {0, 0, 0}, jtr[2] = {0, 0};
        for (int t = 0; t < m; ++t) {
            if (x[t] <= 0.0) continue;   // model 1, no dependence on a or b
            const double p = pow(x[t], 2.0 * b), den = 1.0 + a * p;
            const double r = 1.0 / den - y[t];
            const double ja = -p / (den * den), jb = -a * p * 2.0 * log(x[t]) / (den * den);
            jtj[0] += ja * ja;
            jtj[1] += ja * jb;
            jtj[2] += jb * jb;
            jtr[0] += ja * r;
            jtr[1] += jb * r;
        }
        for (int tries = 0; tries < 60; ++tries) {
            const double m00 = jtj[0] * (1.0 + lam), m11 = jtj[2] * (1.0 + lam), m01 = jtj[1];
            const double det = m00 * m11 - m01 * m01;
            if (!(fabs(det) > 0.0)) { lam *= 10.0; continue; }
            const double da = (-jtr[0] * m11 + jtr[1] * m01) / det;
            const double db = (-jtr[1] * m00 + jtr[0] * m01) / det;
            const double na = a + da, nb = b + db;
            const double ns = (na > 0.0 && nb > 0.0) ? umap_ab_sse(x, y, m, na, nb) : INFINITY;
            if (ns <= sse) {
                const double step = fabs(da) / fabs(a) + fabs(db) / fabs(b);
                a = na;
                b = nb;
                const double gain = sse - ns;
                sse = ns;
                lam = std::max(lam / 10.0, 1e-12);
                if (step < 1e-12 || gain <= 1e-16 * std::max(sse, 1e-300)) done = true;
                break;
            }
            lam *= 10.0;
            if (lam > 1e16) { done = true; break; }
        }
    }
    if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b))
        return fail(RSC_ERR_INVALID_ARG, "a, b fit did not converge");
    *a_out = (float)a;
    *b_out = (float)b;
    return RSC_OK;
}

rsc_status rsc_umap_workspace_size(int64_t n, int64_t nnz, int32_t dim, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    if (n < 1 || n >= (int64_t(1) << 31) || nnz < 0 || nnz >= (int64_t(1) << 31) || dim < 1 || dim > 4)
        return fail(RSC_ERR_INVALID_ARG, "n=%lld, nnz=%lld, dim=%d", (long long)n, (long long)nnz, dim);
    carve_umap(nullptr, n, nnz, dim, bytes);
    return RSC_OK;
}

rsc_status rsc_umap_layout(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n,
                           int64_t nnz, int32_t dim, float *embedding, const rsc_umap_opts *o,
                           void *workspace, size_t workspace_bytes) {
    RSC_TRACE("rsc_umap_layout");
    size_t need = 0;
    rsc_status s = rsc_umap_workspace_size(n, nnz, dim, &need);
    if (s != RSC_OK) return s;
    if (!o) return fail(RSC_ERR_INVALID_ARG, "opts is NULL");
    if (!indptr || !embedding || (nnz > 0 && (!indices || !data)))
        return fail(RSC_ERR_INVALID_ARG, "NULL graph or embedding pointer");
    const int N = o->n_epochs;
    if (N < 1 || N > 100000) return fail(RSC_ERR_INVALID_ARG, "n_epochs=%d out of [1, 100000]", N);
    const int first = o->epoch_first == 0 ? 1 : o->epoch_first;
    const int last = o->epoch_last == 0 ? N : o->epoch_last;
    if (first < 1 || last > N || first > last)
        return fail(RSC_ERR_INVALID_ARG, "epochs %d..%d outside 1..%d", first, last, N);
    if (o->negative_sample_rate < 0 || o->negative_sample_rate > 64)
        return fail(RSC_ERR_INVALID_ARG, "negative_sample_rate=%d out of [0, 64]", o->negative_sample_rate);
    if (!std::isfinite(o->a) || !std::isfinite(o->b) || !std::isfinite(o->gamma) || !std::isfinite(o->learning_rate))
        return fail(RSC_ERR_INVALID_ARG, "non-finite a, b, gamma or learning_rate");
    if ((s = check_ws(workspace, workspace_bytes, need)) != RSC_OK) return s;
    UmapLayout L = carve_umap(workspace, n, nnz, dim, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(o->stream);
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, kStatusBytes, st));
    RSC_CUDA_TRY(launch_umap_prepare(indptr, data, n, nnz, L.wmax, L.f, L.rowoff, st));
    UmapParams p{o->a, o->b, o->gamma, o->learning_rate, o->negative_sample_rate, N, o->seed};
    RSC_CUDA_TRY(launch_umap_epochs(indptr, indices, L.f, L.rowoff, n, nnz, dim, embedding, L.buf0, L.buf1, first,
                                    last, p, L.status, st));
    return RSC_OK;
}

}  // extern "C"
