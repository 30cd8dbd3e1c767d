// Pruned tensor-core candidate search (rows in locality order).
//
// Pass 1 (WindowWork): every query tile scans only the database tiles of its
// own window (its neighbourhood after the locality ordering) and saves each
// (row, part) list, keys and ids, to a state buffer.
// Between the passes (prune.cu) a bounding-sphere test per (query tile,
// database tile) pair keeps only the tiles that can still hold a value below
// some list's saved threshold.
// Pass 2 (ListWork): every query tile resumes its saved lists and scans its
// kept tiles in ascending order (largest lists first across the launch).
//
// The unpruned scan visits the window first and then the other tiles in
// ascending order; a dropped tile's values all lie at or above every
// threshold its query tile reached after the window, and thresholds only
// decrease, so the unpruned scan rejects each of them.  The lists, and the
// candidates, are therefore exactly those of the unpruned scan.
#include "knn_tc.cuh"

namespace rsc {
namespace tck {

// Pass 1: query tile it scans database tiles [lo, hi) around its position.
struct WindowWork {
    static constexpr int kShort = 0;
    static constexpr bool kResume = false;
    static constexpr bool kHitHeavy = true;   // nearby tiles: most of them improve some list
    static constexpr bool kStartBelow = true;     // first tile = the query tile's own
    static constexpr bool kDynamic = false;   // every item scans the same few tiles
    int64_t n;
    int window;
    float *st_key;     // [n, EG, KCP]
    int32_t *st_id;    // [n, EG, KCP]
    int n_items;

    int64_t count_host() const { return n_items; }
    __device__ __forceinline__ int count() const { return n_items; }
    __device__ __forceinline__ WorkItem get(int it) const {
        WorkItem w;
        w.q0 = (int64_t)it * BM;
        w.q_end = min(n, w.q0 + BM);
        const int T = (int)((n + BN - 1) / BN);
        const int tq = (int)(w.q0 / BN);
        const int lo = max(0, tq - window), hi = min(T, tq + window + 1);
        w.j_begin = (int64_t)lo * BN;
        w.j_end = min(n, (int64_t)hi * BN);
        w.tag = 0;
        w.short_list = false;
        w.win_lo = 0;              // the whole range is the window, from the centre
        w.win_hi = hi - lo;
        w.win_c = tq - lo;
        w.tiles = nullptr;
        w.n_tiles = 0;
        w.skip_window = false;
        return w;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &, int part, int64_t q, const RowTopK<KCP> &list) const {
        const int64_t base = (q * EG + part) * KCP;
#pragma unroll
        for (int c = 0; c < KCP; ++c) {
            st_key[base + c] = list.key[c];
            st_id[base + c] = list.id[c];
        }
    }
};

// Pass 2: resume the saved lists, scan the kept tiles, emit candidate ids.
// When the kept-tile lists overflowed their buffer (*overflow != 0) every
// tile outside the window is scanned instead.
struct ListWork {
    static constexpr int kShort = 0;
    static constexpr bool kResume = true;
    static constexpr bool kHitHeavy = true;   // nearby tiles: most of them improve some list
    static constexpr bool kStartBelow = false;
    static constexpr bool kDynamic = true;    // kept-tile counts differ widely between query tiles
    int64_t n;
    int window;
    const float *st_key;
    const int32_t *st_id;
    const int32_t *tiles;       // kept tiles, query tile after query tile (ascending)
    const int64_t *tile_off;    // [n_items + 1]
    const int32_t *order;       // [n_items]: query tiles, largest kept-tile count first
    const int32_t *overflow;    // [1]
    int32_t *cand;              // [EG, n, KCP]
    int n_items;
    int *counter;               // next item (zeroed before the launch)

    int64_t count_host() const { return n_items; }
    __device__ __forceinline__ int count() const { return n_items; }
    __device__ __forceinline__ WorkItem get(int pos) const {
        const int it = order[pos];
        WorkItem w;
        w.q0 = (int64_t)it * BM;
        w.q_end = min(n, w.q0 + BM);
        w.j_begin = 0;
        w.j_end = n;
        w.tag = 0;
        w.short_list = false;
        w.win_lo = w.win_hi = w.win_c = 0;
        w.skip_window = false;
        if (*overflow == 0) {
            w.tiles = tiles + tile_off[it];
            w.n_tiles = (int)(tile_off[it + 1] - tile_off[it]);
        } else {
            w.tiles = nullptr;   // fallback: the window is already in the lists, scan the rest
            w.n_tiles = 0;
            const int T = (int)((n + BN - 1) / BN);
            const int tq = (int)(w.q0 / BN);
            w.win_lo = max(0, tq - window);
            w.win_hi = min(T, tq + window + 1);
            w.win_c = tq;
            w.skip_window = true;
        }
        return w;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void resume(const WorkItem &, int part, int64_t q, RowTopK<KCP> &list) const {
        const int64_t base = (q * EG + part) * KCP;
#pragma unroll
        for (int c = 0; c < KCP; ++c) {
            list.key[c] = st_key[base + c];
            list.id[c] = st_id[base + c];
        }
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &, int part, int64_t q, const RowTopK<KCP> &list) const {
        int32_t *out = cand + ((int64_t)part * n + q) * KCP;
#pragma unroll
        for (int c = 0; c < KCP; ++c) out[c] = list.id[c];
    }
};

}  // namespace tck

cudaError_t launch_knn_tc_window(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh,
                                 int window, float *st_key, int32_t *st_id, unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, n, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, n, 1, tck::BN)) != cudaSuccess) return e;
    tck::WindowWork work{n, window, st_key, st_id, (int)ceil_div(n, tck::BM)};
#define RSC_TC_CASE(kcp, eg) return tck::launch_kernel<1, kcp, eg>(mq, md, work, status, st, sh.stages)
    if (sh.parts == 4 && sh.list == 16) RSC_TC_CASE(16, 4);
    if (sh.parts == 2 && sh.list == 16) RSC_TC_CASE(16, 2);
    if (sh.parts == 2 && sh.list == 32) RSC_TC_CASE(32, 2);
    if (sh.parts == 2 && sh.list == 64) RSC_TC_CASE(64, 2);
#undef RSC_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_knn_tc_list(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh, int window,
                               const float *st_key, const int32_t *st_id, const int32_t *tiles,
                               const int64_t *tile_off, const int32_t *order, const int32_t *overflow,
                               int32_t *cand, int *counter, unsigned int *status, cudaStream_t st) {
    if (tc_kb(d, metric) != 1) return cudaErrorInvalidValue;
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, n, 1, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, n, 1, tck::BN)) != cudaSuccess) return e;
    tck::ListWork work{n, window, st_key, st_id, tiles, tile_off, order, overflow, cand, (int)ceil_div(n, tck::BM), counter};
    if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
#define RSC_TC_CASE(kcp, eg) return tck::launch_kernel<1, kcp, eg>(mq, md, work, status, st, sh.stages)
    if (sh.parts == 4 && sh.list == 16) RSC_TC_CASE(16, 4);
    if (sh.parts == 2 && sh.list == 16) RSC_TC_CASE(16, 2);
    if (sh.parts == 2 && sh.list == 32) RSC_TC_CASE(32, 2);
    if (sh.parts == 2 && sh.list == 64) RSC_TC_CASE(64, 2);
#undef RSC_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rsc
