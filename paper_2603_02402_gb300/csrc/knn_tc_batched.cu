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

namespace rsc {

namespace tck {

struct BatchedWork {
    static constexpr int kShort = 4;   // ids kept per (query, sample, part) for cross lists
    static constexpr bool kResume = false;
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
        w.win_lo = w.win_hi = 0;
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

}  // namespace tck

namespace {

constexpr int kXWarps = 4;

__device__ __forceinline__ bool pair_gt(float ka, int ia, float kb, int ib) {
    return ka > kb || (ka == kb && ia > ib);
}

// One warp per query: for every sample, re-score its 16 cross candidates
// exactly (direct difference in FP32), keep the k_cross best by (distance,
// id), take the own sample's from the exact within lists, then order the
// row's S * k_cross entries by (distance, id).
__global__ void __launch_bounds__(kXWarps * 32)
rerank_cross_kernel(const float *__restrict__ R, int64_t rs, int64_t N, int d, int metric,
                    const int64_t *__restrict__ samp_off, int S, const int32_t *__restrict__ cand_x,
                    const int32_t *__restrict__ idx_w, const float *__restrict__ dist_w, int k_within,
                    int k_cross, int L2, int parts, int32_t *__restrict__ idx_x, float *__restrict__ dist_x) {
    const int n_cand = parts * tck::BatchedWork::kShort;   // candidates per (query, sample)
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int XQ = 65;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xq = reinterpret_cast<float *>(smem) + warp * XQ;
    float *rkey = reinterpret_cast<float *>(smem) + kXWarps * XQ + warp * L2;
    int *rid = reinterpret_cast<int *>(reinterpret_cast<float *>(smem) + kXWarps * XQ + kXWarps * L2) + warp * L2;
    const int64_t q = (int64_t)blockIdx.x * kXWarps + warp;
    if (q >= N) return;
    const bool cosine = metric == RSC_COSINE;
    const int width = cosine ? d + 1 : d;
    for (int t = lane; t < width; t += 32) xq[t] = R[q * rs + t];
    // own sample (binary search in the offsets)
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
            const int32_t j = cand_x[((int64_t)q * S + t) * n_cand + hl];
            if (j >= 0) {
                const float *yr = R + (int64_t)j * rs;
                float acc = 0.f;
                for (int u = 0; u < d; ++u) {
                    const float diff = xq[u] - __ldg(yr + u);
                    acc = fmaf(diff, diff, acc);
                }
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
        rkey[own * k_cross + c] = dist_w[q * k_within + c];
        rid[own * k_cross + c] = idx_w[q * k_within + c];
    }
    __syncwarp();
    // order the whole row by (distance, id)
    for (int size = 2; size <= L2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < L2 / 2; i += 32) {
                const int a = (i / stride) * 2 * stride + (i % stride), b = a + stride;
                const bool asc = (a & size) == 0;
                const float ka = rkey[a], kb = rkey[b];
                const int ia = rid[a], ib = rid[b];
                if (asc ? pair_gt(ka, ia, kb, ib) : pair_gt(kb, ib, ka, ia)) {
                    rkey[a] = kb;
                    rkey[b] = ka;
                    rid[a] = ib;
                    rid[b] = ia;
                }
            }
            __syncwarp();
        }
    }
    const int W = S * k_cross;
    for (int c = lane; c < W; c += 32) {
        const bool valid = rid[c] != INT_MAX;
        idx_x[q * W + c] = valid ? rid[c] : -1;
        dist_x[q * W + c] = valid ? rkey[c] : INFINITY;
    }
}

}  // namespace

// Host-built tables, uploaded once per call: tile_row[T], tile_end[T],
// samp_off[S + 1] (int64), tile_samp[T], samp_order[S], item counter (int32,
// uploaded as 0).
size_t batched_tables_bytes(int T, int S) {
    return sizeof(int64_t) * (2 * (size_t)T + S + 1) + sizeof(int32_t) * ((size_t)T + S + 1);
}

int64_t batched_query_tiles(const int64_t *offsets_host, int S) {
    int64_t T = 0;
    for (int s = 0; s < S; ++s) T += ceil_div(offsets_host[s + 1] - offsets_host[s], tck::BM);
    return T;
}

// Host tables: tile_row [T], tile_end [T], samp_off [S+1], tile_samp [T] (in this order).
void batched_fill_tables(const int64_t *offsets_host, int S, void *host_buf) {
    const int64_t T = batched_query_tiles(offsets_host, S);
    int64_t *tile_row = static_cast<int64_t *>(host_buf);
    int64_t *tile_end = tile_row + T;
    int64_t *samp_off = tile_end + T;
    int32_t *tile_samp = reinterpret_cast<int32_t *>(samp_off + S + 1);
    int64_t t = 0;
    for (int s = 0; s < S; ++s) {
        for (int64_t r = offsets_host[s]; r < offsets_host[s + 1]; r += tck::BM) {
            tile_row[t] = r;
            tile_end[t] = std::min<int64_t>(offsets_host[s + 1], r + tck::BM);
            tile_samp[t] = s;
            ++t;
        }
    }
    for (int s = 0; s <= S; ++s) samp_off[s] = offsets_host[s];
    int32_t *samp_order = tile_samp + T;
    for (int s = 0; s < S; ++s) samp_order[s] = s;
    std::stable_sort(samp_order, samp_order + S, [&](int32_t a, int32_t b) {
        return offsets_host[a + 1] - offsets_host[a] > offsets_host[b + 1] - offsets_host[b];
    });
    samp_order[S] = 0;   // the item counter
}

cudaError_t launch_knn_tc_batched(const void *Qb, const void *Db, int64_t N, int d, int metric, int S, int T,
                                  int parts, const void *tables_dev, int32_t *cand_w, int32_t *cand_x,
                                  unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, N, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, N, 1, tck::BN)) != cudaSuccess) return e;
    const int64_t *tile_row = static_cast<const int64_t *>(tables_dev);
    const int64_t *tile_end = tile_row + T;
    const int64_t *samp_off = tile_end + T;
    const int32_t *tile_samp = reinterpret_cast<const int32_t *>(samp_off + S + 1);
    const int32_t *samp_order = tile_samp + T;
    int *counter = const_cast<int *>(samp_order + S);
    tck::BatchedWork work{T, S, tile_row, tile_end, tile_samp, samp_off, N, cand_w, cand_x, samp_order, counter};
    if (parts == 4) return tck::launch_kernel<1, kBatchedList, 4>(mq, md, work, status, st);
    if (parts == 2) return tck::launch_kernel<1, kBatchedList, 2>(mq, md, work, status, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_rerank_cross(const float *R, int64_t rs, int64_t N, int d, int metric, const void *tables_dev,
                                int S, int T, int parts, const int32_t *cand_x, const int32_t *idx_w,
                                const float *dist_w, int k_within, int k_cross, int32_t *idx_x, float *dist_x,
                                cudaStream_t st) {
    if (parts != 2 && parts != 4) return cudaErrorInvalidValue;
    const int64_t *samp_off = static_cast<const int64_t *>(tables_dev) + 2 * (int64_t)T;
    int L2 = 32;
    while (L2 < S * k_cross) L2 <<= 1;
    if (L2 > 1024) return cudaErrorInvalidValue;
    constexpr int XQ = 65;
    const size_t smem = sizeof(float) * kXWarps * XQ + (sizeof(float) + sizeof(int)) * kXWarps * L2;
    rerank_cross_kernel<<<(unsigned)ceil_div(N, kXWarps), kXWarps * 32, smem, st>>>(
        R, rs, N, d, metric, samp_off, S, cand_x, idx_w, dist_w, k_within, k_cross, L2, parts, idx_x, dist_x);
    return cudaGetLastError();
}

}  // namespace rsc
