// Batched kNN over many samples in one persistent tensor-core launch.
//
// Cells are grouped by sample through category offsets (the CSR-like
// category-index mapping the paper uses for its group-pair kernels, Methods,
// "Perturbation distance computation").  For every cell the launch finds
//   * its k_within nearest cells inside its own sample, and
//   * the k_cross nearest cells from every sample (own included): the
//     batch-balanced neighbour lists consumed by batch-aware graphs.
// Work items are (query tile of one sample, database sample) pairs; a tile
// never straddles two samples, so an item either is "within" (database sample
// = the tile's own sample, full lists kept) or "cross" (only the best
// kShort of each part list are needed and kept).  Items are ordered database
// sample first, so the CTAs of a wave stream the same sample from L2.
// Both candidate sets are re-scored exactly in FP32 (rerank.cu for within,
// rerank_cross_kernel below for cross).
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "knn_tc.cuh"
#include "warp_sort.cuh"

namespace rsc {

namespace tck {

struct BatchedWork {
    static constexpr int kShort = 4;   // ids kept per (query, sample, part) for cross lists
    static constexpr bool kResume = false;
    static constexpr bool kHitHeavy = false;
    static constexpr bool kStartBelow = false;
    static constexpr bool kDynamic = true;   // item cost follows its database sample's size
    int T;                             // query tiles
    int S;                             // samples
    const int64_t *tile_row;           // [T] first row of the tile
    const int64_t *tile_end;           // [T] one past its last row (inside its sample)
    const int32_t *tile_samp;          // [T] its sample
    const int64_t *samp_off;           // [S + 1]
    int64_t N;
    int32_t *cand_w;                   // [EG, N, KCP]      within-sample lists
    int32_t *cand_x;                   // [N, S, EG, kShort] cross-sample lists
    const int32_t *samp_order;         // [S] samples by decreasing size (largest items first)
    int *counter;                      // next item (zeroed by the table upload)

    int64_t count_host() const { return (int64_t)T * S; }
    __device__ __forceinline__ int count() const { return T * S; }
    __device__ __forceinline__ WorkItem get(int it) const {
        const int r = it / T, qt = it - r * T;
        const int t = samp_order[r];
        WorkItem w;
        w.q0 = tile_row[qt];
        w.q_end = tile_end[qt];
        w.j_begin = samp_off[t];
        w.j_end = samp_off[t + 1];
        w.tag = t;
        w.short_list = tile_samp[qt] != t;
        w.win_lo = w.win_hi = w.win_c = 0;
        w.tiles = nullptr;
        w.n_tiles = 0;
        w.skip_window = false;
        return w;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &w, int part, int64_t q, const RowTopK<KCP> &list) const {
        if (!w.short_list) {
            int32_t *out = cand_w + ((int64_t)part * N + q) * KCP;
#pragma unroll
            for (int c = 0; c < KCP; ++c) out[c] = list.id[c];
        } else {
            int32_t *out = cand_x + (((int64_t)q * S + w.tag) * EG + part) * kShort;
#pragma unroll
            for (int c = 0; c < kShort; ++c) out[c] = list.id[c];
        }
    }
};

// Pruned batched search (rows in locality order inside each sample).
// Pass 1: item (query tile qt, sample t) scans only the tiles of sample t
// around win[t * T + qt], the tile of t whose bounding-sphere centre is
// nearest the query tile's, and saves its lists (keys in st_w / st_x, ids in
// cand_w / cand_x).
struct BatchedWindowWork {
    static constexpr int kShort = kBatchedShort;
    static constexpr bool kResume = false;
    static constexpr bool kHitHeavy = true;   // nearby tiles: most of them improve some list
    static constexpr bool kStartBelow = true;     // first tile = the nearest of the sample
    static constexpr bool kDynamic = true;
    int T, S;
    const int64_t *tile_row, *tile_end;
    const int32_t *tile_samp;
    const int64_t *samp_off;
    const int32_t *samp_order;
    int *counter;
    int64_t N;
    const int32_t *win;
    int window;
    float *st_w;
    int32_t *cand_w;
    float *st_x;
    int32_t *cand_x;

    int64_t count_host() const { return (int64_t)T * S; }
    __device__ __forceinline__ int count() const { return T * S; }
    __device__ __forceinline__ WorkItem get(int it) const {
        const int r = it / T, qt = it - r * T;
        const int t = samp_order[r];
        const int64_t b = samp_off[t], e = samp_off[t + 1];
        const int Tt = (int)((e - b + BN - 1) / BN);
        const int w = win[(int64_t)t * T + qt];
        const int lo = max(0, w - window), hi = min(Tt, w + window + 1);
        WorkItem wi;
        wi.q0 = tile_row[qt];
        wi.q_end = tile_end[qt];
        wi.j_begin = b + (int64_t)lo * BN;
        wi.j_end = min(e, b + (int64_t)hi * BN);
        wi.tag = t;
        wi.short_list = tile_samp[qt] != t;
        wi.win_lo = 0;             // the whole range is the window, from the centre
        wi.win_hi = hi - lo;
        wi.win_c = w - lo;
        wi.tiles = nullptr;
        wi.n_tiles = 0;
        wi.skip_window = false;
        return wi;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &w, int part, int64_t q, const RowTopK<KCP> &list) const {
        if (!w.short_list) {
            const int64_t base = ((int64_t)part * N + q) * KCP;
#pragma unroll
            for (int c = 0; c < KCP; ++c) {
                st_w[base + c] = list.key[c];
                cand_w[base + c] = list.id[c];
            }
        } else {
            const int64_t base = (((int64_t)q * S + w.tag) * EG + part) * kShort;
#pragma unroll
            for (int c = 0; c < kShort; ++c) {
                st_x[base + c] = list.key[c];
                cand_x[base + c] = list.id[c];
            }
        }
    }
};

// Pass 2: resume the saved lists and scan the kept tiles of sample t
// (local tile indices, ascending, window excluded); if the kept-tile lists
// overflowed their buffer, every tile of t outside the window instead.
struct BatchedListWork {
    static constexpr int kShort = kBatchedShort;
    static constexpr bool kResume = true;
    static constexpr bool kHitHeavy = true;   // nearby tiles: most of them improve some list
    static constexpr bool kStartBelow = false;
    static constexpr bool kDynamic = true;
    int T, S;
    const int64_t *tile_row, *tile_end;
    const int32_t *tile_samp;
    const int64_t *samp_off;
    const int32_t *samp_order;
    int *counter;
    int64_t N;
    const int32_t *win;
    int window;
    const float *st_w;
    int32_t *cand_w;
    const float *st_x;
    int32_t *cand_x;
    const int32_t *tiles;
    const int64_t *tile_off;    // [T * S + 1], item t * T + qt
    const int32_t *overflow;

    int64_t count_host() const { return (int64_t)T * S; }
    __device__ __forceinline__ int count() const { return T * S; }
    __device__ __forceinline__ WorkItem get(int it) const {
        const int r = it / T, qt = it - r * T;
        const int t = samp_order[r];
        const int64_t item = (int64_t)t * T + qt;
        WorkItem wi;
        wi.q0 = tile_row[qt];
        wi.q_end = tile_end[qt];
        wi.j_begin = samp_off[t];
        wi.j_end = samp_off[t + 1];
        wi.tag = t;
        wi.short_list = tile_samp[qt] != t;
        wi.win_lo = wi.win_hi = wi.win_c = 0;
        wi.skip_window = false;
        if (*overflow == 0) {
            wi.tiles = tiles + tile_off[item];
            wi.n_tiles = (int)(tile_off[item + 1] - tile_off[item]);
        } else {
            const int Tt = (int)((wi.j_end - wi.j_begin + BN - 1) / BN);
            const int w = win[item];
            wi.tiles = nullptr;
            wi.n_tiles = 0;
            wi.win_lo = max(0, w - window);
            wi.win_hi = min(Tt, w + window + 1);
            wi.win_c = w;
            wi.skip_window = true;
        }
        return wi;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void resume(const WorkItem &w, int part, int64_t q, RowTopK<KCP> &list) const {
        if (!w.short_list) {
            const int64_t base = ((int64_t)part * N + q) * KCP;
#pragma unroll
            for (int c = 0; c < KCP; ++c) {
                list.key[c] = st_w[base + c];
                list.id[c] = cand_w[base + c];
            }
        } else {
            const int64_t base = (((int64_t)q * S + w.tag) * EG + part) * kShort;
#pragma unroll
            for (int c = 0; c < kShort; ++c) {
                list.key[c] = st_x[base + c];
                list.id[c] = cand_x[base + c];
            }
        }
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &w, int part, int64_t q, const RowTopK<KCP> &list) const {
        if (!w.short_list) {
            int32_t *out = cand_w + ((int64_t)part * N + q) * KCP;
#pragma unroll
            for (int c = 0; c < KCP; ++c) out[c] = list.id[c];
        } else {
            int32_t *out = cand_x + (((int64_t)q * S + w.tag) * EG + part) * kShort;
#pragma unroll
            for (int c = 0; c < kShort; ++c) out[c] = list.id[c];
        }
    }
};

}  // namespace tck

namespace {

constexpr int kXWarps = 4;

// One warp per query position q (original row qo = perm[q], or q without a
// permutation): for every sample, re-score its cross candidates exactly
// (direct difference in FP32), keep the k_cross best by (distance, id), take
// the own sample's from the exact within lists, then order the row's
// S * k_cross entries by (distance, id) with a register bitonic network
// (E = L2 / 32 entries per lane).  Candidate ids are positions, mapped to
// original rows through perm; R holds the rows by position when r_by_pos.
template <int E>
__global__ void __launch_bounds__(kXWarps * 32)
rerank_cross_kernel(const float *__restrict__ R, int64_t rs, int64_t N, int d, int metric, int w4,
                    const int64_t *__restrict__ samp_off, int S, const int32_t *__restrict__ cand_x,
                    const int32_t *__restrict__ perm, bool r_by_pos, const int32_t *__restrict__ idx_w,
                    const float *__restrict__ dist_w, int k_within, int k_cross, int parts,
                    int32_t *__restrict__ idx_x, float *__restrict__ dist_x) {
    constexpr int L2 = 32 * E;
    const int n_cand = parts * tck::BatchedWork::kShort;   // candidates per (query, sample)
    __shared__ __align__(16) float xq_s[kXWarps][68];
    __shared__ float rkey_s[kXWarps][L2];
    __shared__ int rid_s[kXWarps][L2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xq = xq_s[warp];
    float *rkey = rkey_s[warp];
    int *rid = rid_s[warp];
    const int64_t q = (int64_t)blockIdx.x * kXWarps + warp;
    if (q >= N) return;
    const int64_t qo = perm ? (int64_t)perm[q] : q;
    const int64_t qr = r_by_pos ? q : qo;
    const bool cosine = metric == RSC_COSINE;
    const int width = cosine ? d + 1 : d;
    for (int t = lane; t < width; t += 32) xq[t] = R[qr * rs + t];
    // own sample (binary search in the offsets; positions keep the sample ranges)
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (samp_off[mid] <= q) lo = mid;
        else hi = mid;
    }
    const int own = lo;
    for (int e = lane; e < L2; e += 32) {
        rkey[e] = INFINITY;
        rid[e] = INT_MAX;
    }
    __syncwarp();
    const bool fq = cosine && xq[d] != 0.f;
    // two samples per pass: lanes 0-15 sample t, lanes 16-31 sample t + 1
    // (lanes past n_cand hold +inf)
    const int half = lane >> 4, hl = lane & 15;
    for (int t0 = 0; t0 < S; t0 += 2) {
        const int t = t0 + half;
        float key = INFINITY;
        int id = INT_MAX;
        if (t < S && t != own && hl < n_cand) {
            const int32_t jp = cand_x[((int64_t)q * S + t) * n_cand + hl];
            if (jp >= 0 && (int64_t)jp < N) {   // ids outside [0, N) (an aborted search) are skipped
                const int32_t j = perm ? perm[jp] : jp;
                const float *yr = R + (int64_t)(r_by_pos ? jp : j) * rs;
                float acc = row_dist2(xq, yr, d, w4);
                if (cosine) {
                    const bool fy = __ldg(yr + d) != 0.f;
                    if (fq || fy) acc = (fq && fy) ? 0.f : 2.f;
                }
                key = cosine ? 0.5f * acc : sqrtf(acc);
                id = j;
            }
        }
        // sort each 16-lane half ascending by (key, id): bitonic over lanes
#pragma unroll
        for (int size = 2; size <= 16; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const float ok = __shfl_xor_sync(0xffffffffu, key, stride);
                const int oi = __shfl_xor_sync(0xffffffffu, id, stride);
                const bool up = (hl & size) == 0;          // this block sorts ascending
                const bool lower = (hl & stride) == 0;     // this lane is the lower of the pair
                const bool keep_min = (lower == up);
                const bool take = keep_min ? pair_gt(key, id, ok, oi) : pair_gt(ok, oi, key, id);
                if (take) {
                    key = ok;
                    id = oi;
                }
            }
        }
        if (t < S && t != own && hl < k_cross) {
            rkey[t * k_cross + hl] = key;
            rid[t * k_cross + hl] = id;
        }
    }
    // own sample: the first k_cross of the exact within list
    for (int c = lane; c < k_cross; c += 32) {
        rkey[own * k_cross + c] = dist_w[qo * k_within + c];
        rid[own * k_cross + c] = idx_w[qo * k_within + c];
    }
    __syncwarp();
    // order the whole row by (distance, id)
    float key[E];
    int id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        key[e] = rkey[e * 32 + lane];
        id[e] = rid[e * 32 + lane];
    }
    warp_sort_pairs<E>(key, id);
    const int W = S * k_cross;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = e * 32 + lane;
        if (c < W) {
            const bool valid = id[e] != INT_MAX;
            idx_x[qo * W + c] = valid ? id[e] : -1;
            dist_x[qo * W + c] = valid ? key[e] : INFINITY;
        }
    }
}

}  // namespace

// Host-built tables, uploaded once per call (BatchedTables in kernels.h):
// int64 tile_row[T], tile_end[T], samp_off[S + 1], dtile_start[DT],
// dtile_end[DT]; int32 tile_samp[T], samp_order[S], item counter (uploaded
// as 0), dtile_off[S + 1].  Query tiles are 128 rows inside one sample;
// database tiles are 256 rows inside one sample (sample t's tiles are
// dtile_off[t] .. dtile_off[t + 1]).
BatchedTables batched_tables(void *base, int64_t T, int S, int64_t DT) {
    BatchedTables b;
    int64_t *p64 = static_cast<int64_t *>(base);
    b.tile_row = p64;
    b.tile_end = b.tile_row + T;
    b.samp_off = b.tile_end + T;
    b.dtile_start = b.samp_off + S + 1;
    b.dtile_end = b.dtile_start + DT;
    int32_t *p32 = reinterpret_cast<int32_t *>(b.dtile_end + DT);
    b.tile_samp = p32;
    b.samp_order = b.tile_samp + T;
    b.counter = b.samp_order + S;
    b.dtile_off = b.counter + 1;
    return b;
}

size_t batched_tables_bytes(int64_t T, int S, int64_t DT) {
    return sizeof(int64_t) * (2 * (size_t)T + S + 1 + 2 * (size_t)DT) + sizeof(int32_t) * ((size_t)T + S + 1 + S + 1);
}

int64_t batched_query_tiles(const int64_t *offsets_host, int S) {
    int64_t T = 0;
    for (int s = 0; s < S; ++s) T += ceil_div(offsets_host[s + 1] - offsets_host[s], tck::BM);
    return T;
}

int64_t batched_db_tiles(const int64_t *offsets_host, int S) {
    int64_t DT = 0;
    for (int s = 0; s < S; ++s) DT += ceil_div(offsets_host[s + 1] - offsets_host[s], tck::BN);
    return DT;
}

void batched_fill_tables(const int64_t *offsets_host, int S, void *host_buf) {
    const int64_t T = batched_query_tiles(offsets_host, S), DT = batched_db_tiles(offsets_host, S);
    BatchedTables b = batched_tables(host_buf, T, S, DT);
    int64_t t = 0, g = 0;
    for (int s = 0; s < S; ++s) {
        for (int64_t r = offsets_host[s]; r < offsets_host[s + 1]; r += tck::BM) {
            b.tile_row[t] = r;
            b.tile_end[t] = std::min<int64_t>(offsets_host[s + 1], r + tck::BM);
            b.tile_samp[t] = s;
            ++t;
        }
        b.dtile_off[s] = (int32_t)g;
        for (int64_t r = offsets_host[s]; r < offsets_host[s + 1]; r += tck::BN) {
            b.dtile_start[g] = r;
            b.dtile_end[g] = std::min<int64_t>(offsets_host[s + 1], r + tck::BN);
            ++g;
        }
    }
    b.dtile_off[S] = (int32_t)g;
    for (int s = 0; s <= S; ++s) b.samp_off[s] = offsets_host[s];
    for (int s = 0; s < S; ++s) b.samp_order[s] = s;
    std::stable_sort(b.samp_order, b.samp_order + S, [&](int32_t a, int32_t c) {
        return offsets_host[a + 1] - offsets_host[a] > offsets_host[c + 1] - offsets_host[c];
    });
    *b.counter = 0;
}

cudaError_t launch_knn_tc_batched(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                  int64_t DT, int parts, int stages, const void *tables_dev, int32_t *cand_w, int32_t *cand_x,
                                  unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, N, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, N, 1, tck::BN)) != cudaSuccess) return e;
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    tck::BatchedWork work{T,     S, b.tile_row, b.tile_end, b.tile_samp, b.samp_off, N, cand_w, cand_x,
                          b.samp_order, b.counter};
    if (parts == 4) return tck::launch_kernel<1, kBatchedList, 4>(mq, md, work, status, st, stages);
    if (parts == 2) return tck::launch_kernel<1, kBatchedList, 2>(mq, md, work, status, st, stages);
    return cudaErrorInvalidValue;
}

cudaError_t launch_rerank_cross(const float *R, int64_t rs, int64_t N, int d, int metric, const void *tables_dev,
                                int S, int T, int64_t DT, int parts, const int32_t *cand_x, const int32_t *perm,
                                bool r_by_pos, const int32_t *idx_w, const float *dist_w, int k_within, int k_cross,
                                int32_t *idx_x, float *dist_x, cudaStream_t st) {
    if (parts != 2 && parts != 4) return cudaErrorInvalidValue;
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    int L2 = 32;
    while (L2 < S * k_cross) L2 <<= 1;
    const int width = metric == RSC_COSINE ? d + 1 : d;
    const bool vec = rs % 4 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0 && width <= 64;
    const int w4 = vec ? (width + 3) / 4 : 0;
    const unsigned blocks = (unsigned)ceil_div(N, kXWarps);
#define RSC_RX(e)                                                                                                 \
    case 32 * e:                                                                                                  \
        rerank_cross_kernel<e><<<blocks, kXWarps * 32, 0, st>>>(R, rs, N, d, metric, w4, b.samp_off, S, cand_x, \
                                                                perm, r_by_pos, idx_w, dist_w, k_within, k_cross, \
                                                                parts, idx_x, dist_x);                            \
        break
    switch (L2) {
        RSC_RX(1); RSC_RX(2); RSC_RX(4); RSC_RX(8); RSC_RX(16); RSC_RX(32);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_RX
    return cudaGetLastError();
}


cudaError_t launch_knn_tc_batched_window(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                         int64_t DT, int parts, int stages, const void *tables_dev, const int32_t *win, int window,
                                         float *st_w, int32_t *cand_w, float *st_x, int32_t *cand_x,
                                         unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, N, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, N, 1, tck::BN)) != cudaSuccess) return e;
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    if ((e = cudaMemsetAsync(b.counter, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    tck::BatchedWindowWork work{T, S, b.tile_row, b.tile_end, b.tile_samp, b.samp_off, b.samp_order, b.counter, N,
                                win, window, st_w, cand_w, st_x, cand_x};
    if (parts == 4) return tck::launch_kernel<1, kBatchedList, 4>(mq, md, work, status, st, stages);
    if (parts == 2) return tck::launch_kernel<1, kBatchedList, 2>(mq, md, work, status, st, stages);
    return cudaErrorInvalidValue;
}

cudaError_t launch_knn_tc_batched_list(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                       int64_t DT, int parts, int stages, const void *tables_dev, const int32_t *win, int window,
                                       const float *st_w, int32_t *cand_w, const float *st_x, int32_t *cand_x,
                                       const int32_t *tiles, const int64_t *tile_off, const int32_t *overflow,
                                       unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, N, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, N, 1, tck::BN)) != cudaSuccess) return e;
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    if ((e = cudaMemsetAsync(b.counter, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    tck::BatchedListWork work{T,      S,     b.tile_row, b.tile_end, b.tile_samp, b.samp_off, b.samp_order,
                              b.counter, N,  win,        window,     st_w,        cand_w,     st_x,
                              cand_x, tiles, tile_off,   overflow};
    if (parts == 4) return tck::launch_kernel<1, kBatchedList, 4>(mq, md, work, status, st, stages);
    if (parts == 2) return tck::launch_kernel<1, kBatchedList, 2>(mq, md, work, status, st, stages);
    return cudaErrorInvalidValue;
}

}  // namespace rsc
