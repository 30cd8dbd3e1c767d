// Approximate kNN by NN-descent (Dong, Charikar & Li, WWW 2011), the method of
// the PyNNDescent search the paper runs on the CPU (Methods, "Benchmarking").
// A neighbour of a neighbour is probably a neighbour: every iteration joins,
// around each point v, the points v's list and reverse list name, and offers
// each joined pair to both endpoints' lists.
//
// This is the synchronous, deterministic form (rsc.h states it in full):
//   init    lists of k: the point itself and k - 1 hashed draws (SplitMix64),
//           ordered by key = (FP32 squared distance bits) << 32 | id;
//   sample  per point, the first S entries flagged new become the forward new
//           sample (flags cleared), the old entries the forward old sample;
//           each sample entry w receives the point's (priority, id) key in
//           reverse slot hash(point) of w by a 64-bit atomicMin, so a slot
//           keeps its smallest key whatever the order of the atomics;
//   join    block per point v: the join lists (forward samples and reverse
//           slots, deduplicated), their rows staged transposed in shared
//           memory, every pair's squared distance by t-ordered fused
//           multiply-adds (the same bits as any sequential evaluation), and
//           each pair offered to both endpoints' candidate slots (hash of the
//           candidate id, 64-bit atomicMin) when it beats the endpoint's last
//           key;
//   merge   warp per point: its list and its candidates ranked together by
//           counting (no sort), the k smallest distinct keys kept, changes
//           counted; the point's slots are cleared for the next iteration.
// Every decision depends only on keys and on minima, so the lists are the
// same bits on every run and equal the oracle's.  An iteration runs only if
// every earlier one changed at least ceil(delta n k) entries, which every
// kernel reads from the change counters on the device (no host round trip).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace nnd {

constexpr uint64_t kEmpty = ~0ull;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;   // SplitMix64 state increment
constexpr int kMaxK = 64;
constexpr int kMaxSlots = 64;
constexpr int kMaxIters = 64;
constexpr int kJoinThreads = 128;
constexpr int kPairSlots = 64;   // per-iteration pair counters, spread over slots

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + i * kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Fibonacci hashing of an id into 2^bits slots.
__device__ __forceinline__ uint32_t slot_of(uint32_t id, int bits) {
    return bits == 0 ? 0u : (id * 0x9E3779B1u) >> (32 - bits);
}

__device__ __forceinline__ uint64_t make_key(float d2, uint32_t id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | id;
}

// Squared distance of rows a and b, accumulated in t order.
__device__ __forceinline__ float row_delta2(const float *__restrict__ X, int d, int64_t a, int64_t b) {
    const float *xa = X + a * d, *xb = X + b * d;
    float acc = 0.f;
    for (int t = 0; t < d; ++t) {
        const float u = __ldg(xa + t) - __ldg(xb + t);
        acc = fmaf(u, u, acc);
    }
    return acc;
}

// Iteration t runs when every earlier iteration changed at least lim entries.
__device__ __forceinline__ bool active(const unsigned long long *__restrict__ ch, int t, long long lim) {
    for (int j = 0; j < t; ++j)
        if ((long long)ch[j] < lim) return false;
    return true;
}

// Ascending bitonic sort of 32 E keys across a warp (element e * 32 + lane).
template <int E>
__device__ __forceinline__ void warp_sort_u64(uint64_t (&v)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int es = stride >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = e ^ es;
                    if (p > e) {
                        const bool asc = (((e << 5) | lane) & size) == 0;
                        if ((v[e] > v[p]) == asc) {
                            const uint64_t x = v[e];
                            v[e] = v[p];
                            v[p] = x;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], stride);
                    const bool asc = (((e << 5) | lane) & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    if ((lower == asc) ? (o < v[e]) : (o > v[e])) v[e] = o;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ init

// Warp per point: lane 0 picks the ids (the caller's list if any, the hashed
// draws, then consecutive points if the draws repeat too often), every lane
// computes the distances of its entries, the warp sorts the keys.
constexpr int kInitWarps = 8;

__global__ void __launch_bounds__(kInitWarps * 32)
init_kernel(const float *__restrict__ X, int64_t n, int d, int k, uint64_t seed, const int32_t *__restrict__ init,
            uint64_t *__restrict__ key, unsigned long long *__restrict__ flags) {
    __shared__ int32_t s_ids[kInitWarps][kMaxK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kInitWarps + warp;
    if (u >= n) return;   // warp-uniform
    int32_t *ids = s_ids[warp];
    if (lane == 0) {
        int m = 0;
        ids[m++] = (int32_t)u;
        if (init)
            for (int c = 0; c < k && m < k; ++c) {
                const int32_t r = init[u * k + c];
                bool seen = r < 0 || (int64_t)r >= n;
                for (int i = 0; i < m; ++i) seen |= ids[i] == r;
                if (!seen) ids[m++] = r;
            }
        for (int j = 0; j < 2 * k && m < k; ++j) {
            const uint64_t g = splitmix64(seed, (uint64_t)u * (uint64_t)(2 * k) + (uint64_t)j + 1);
            const int32_t r = (int32_t)((u + 1 + (int64_t)(g % (uint64_t)(n - 1))) % n);
            bool seen = false;
            for (int i = 0; i < m; ++i) seen |= ids[i] == r;
            if (!seen) ids[m++] = r;
        }
        for (int64_t s = 1; m < k; ++s) {   // ends within n - 1 steps (k <= n)
            const int32_t r = (int32_t)((u + s) % n);
            bool seen = false;
            for (int i = 0; i < m; ++i) seen |= ids[i] == r;
            if (!seen) ids[m++] = r;
        }
    }
    __syncwarp();
    uint64_t v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = e * 32 + lane;
        v[e] = kEmpty;
        if (c < k) v[e] = make_key(row_delta2(X, d, u, ids[c]), (uint32_t)ids[c]);
    }
    warp_sort_u64<2>(v);
    unsigned long long fl = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = e * 32 + lane;
        const bool isnew = c < k && (int64_t)(uint32_t)v[e] != u;
        if (c < k) key[u * k + c] = v[e];
        fl |= (unsigned long long)__ballot_sync(0xffffffffu, isnew) << (32 * e);
    }
    if (lane == 0) flags[u] = fl;
}

// ---------------------------------------------------------------- sample

// Warp per point (entry c = e * 32 + lane): forward samples chosen from the
// flags, reverse keys offered to the sample entries' slots.
constexpr int kSampleWarps = 8;

__global__ void __launch_bounds__(kSampleWarps * 32)
sample_kernel(int64_t n, int k, int S, int lr, uint64_t seed, int t, const unsigned long long *__restrict__ ch,
              long long lim, const uint64_t *__restrict__ key, unsigned long long *__restrict__ flags,
              unsigned long long *__restrict__ smask, unsigned long long *__restrict__ rn,
              unsigned long long *__restrict__ ro) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kSampleWarps + warp;
    if (u >= n || !active(ch, t, lim)) return;   // warp-uniform
    const int R = 1 << lr;
    const unsigned long long fl = flags[u];
    uint32_t id[2];
    unsigned long long self = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = e * 32 + lane;
        id[e] = c < k ? (uint32_t)key[u * k + c] : 0xFFFFFFFFu;
        self |= (unsigned long long)__ballot_sync(0xffffffffu, c < k && (int64_t)id[e] == u) << (32 * e);
    }
    const unsigned long long valid = k == 64 ? ~0ull : ((1ull << k) - 1);
    const unsigned long long nw = fl & ~self;
    const unsigned long long old = valid & ~fl & ~self;
    const uint64_t pr = splitmix64(seed, ((uint64_t)(t + 1) << 40) | (uint64_t)u) >> 32;
    const unsigned long long pk = (pr << 32) | (uint64_t)(uint32_t)u;
    const uint32_t s = slot_of((uint32_t)u, lr);
    unsigned long long sampled = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int c = e * 32 + lane;
        const bool in_new = c < k && ((nw >> c) & 1ull);
        const bool take = in_new && __popcll(nw & ((1ull << c) - 1ull)) < S;
        if (take) atomicMin(rn + (size_t)id[e] * R + s, pk);
        if (c < k && ((old >> c) & 1ull)) atomicMin(ro + (size_t)id[e] * R + s, pk);
        sampled |= (unsigned long long)__ballot_sync(0xffffffffu, take) << (32 * e);
    }
    if (lane == 0) {
        flags[u] = fl & ~sampled;
        smask[u] = sampled;
    }
}

// ------------------------------------------------------------------ join

// Appends the lanes' ids with keep set to list[*count ..) in lane order.
__device__ __forceinline__ void warp_append(bool keep, int32_t id, int32_t *list, int &count) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) list[count + __popc(m & ((1u << lane) - 1u))] = id;
    count += __popc(m);
    __syncwarp();
}

__device__ __forceinline__ bool listed(const int32_t *list, int count, int32_t id) {
    bool f = false;
    for (int i = 0; i < count; ++i) f |= list[i] == id;
    return f;
}

// Block per point v.  Join rows 0 .. a-1 are new(v), a .. a+o-1 old(v);
// s_x holds row r's coordinate t at t * P + r (P odd: the staging stores of
// one row, lanes over t, fall in distinct banks).  Pairs (i, j), i < a,
// j > i, in 2 x 4 register tiles.
__global__ void __launch_bounds__(kJoinThreads)
join_kernel(const float *__restrict__ X, int64_t n, int d, int k, int lr, int lc, int P, int t,
            const unsigned long long *__restrict__ ch, long long lim, const uint64_t *__restrict__ key,
            const unsigned long long *__restrict__ flags, const unsigned long long *__restrict__ smask,
            const unsigned long long *__restrict__ rn, const unsigned long long *__restrict__ ro,
            unsigned long long *__restrict__ cand, unsigned long long *__restrict__ pairs) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_thr = reinterpret_cast<uint64_t *>(smem);       // [P]
    int32_t *s_id = reinterpret_cast<int32_t *>(s_thr + P);     // [P]
    float *s_x = reinterpret_cast<float *>(s_id + P);           // [d][P]
    __shared__ int s_cnt[2];
    const int64_t v = blockIdx.x;
    if (!active(ch, t, lim)) return;   // block-uniform
    const int R = 1 << lr, C = 1 << lc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        // join lists: new = forward new sample + new reverse slots; old =
        // (forward old sample + old reverse slots) minus new; deduplicated
        const unsigned long long sm = smask[v], post = flags[v];
        int32_t id[2];
        bool self[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            id[e] = c < k ? (int32_t)(uint32_t)key[v * k + c] : -1;
            self[e] = (int64_t)id[e] == v;
        }
        int a = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            warp_append(c < k && ((sm >> c) & 1ull), id[e], s_id, a);
        }
        const int a0 = a;
        for (int s0 = 0; s0 < R; s0 += 32) {
            const int s = s0 + lane;
            const unsigned long long q = s < R ? rn[(size_t)v * R + s] : kEmpty;
            const int32_t r = (int32_t)(uint32_t)q;
            warp_append(q != kEmpty && !listed(s_id, a0, r), r, s_id, a);
        }
        int o = 0;
        int32_t *s_old = s_id + a;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            const bool is_old = c < k && !self[e] && !(((post | sm) >> c) & 1ull);
            warp_append(is_old && !listed(s_id, a, id[e]), id[e], s_old, o);
        }
        const int o0 = o;
        for (int s0 = 0; s0 < R; s0 += 32) {
            const int s = s0 + lane;
            const unsigned long long q = s < R ? ro[(size_t)v * R + s] : kEmpty;
            const int32_t r = (int32_t)(uint32_t)q;
            warp_append(q != kEmpty && !listed(s_id, a, r) && !listed(s_old, o0, r), r, s_old, o);
        }
        if (lane == 0) {
            s_cnt[0] = a;
            s_cnt[1] = o;
        }
    }
    __syncthreads();
    const int a = s_cnt[0], m = a + s_cnt[1];
    if (a == 0) return;   // no new entry joins anything (block-uniform)
    if (threadIdx.x == 0)  // pairs joined (a statistic: rsc_knn_descent_pairs)
        atomicAdd(pairs + t * kPairSlots + (blockIdx.x & (kPairSlots - 1)),
                  (unsigned long long)a * (a - 1) / 2 + (unsigned long long)a * (m - a));
    // stage the rows: each warp takes four rows at a time, all their loads
    // issued before the stores
    const int nwarps = kJoinThreads / 32;
    for (int r0 = 4 * warp; r0 < m; r0 += 4 * nwarps) {
        float v[4][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + q;
            const float *xr = X + (int64_t)(r < m ? s_id[r] : 0) * d;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int tt = lane + 32 * h;
                v[q][h] = (r < m && tt < d) ? __ldg(xr + tt) : 0.f;
            }
        }
        if (lane < 4 && r0 + lane < m) s_thr[r0 + lane] = key[(int64_t)s_id[r0 + lane] * k + k - 1];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int tt = lane + 32 * h;
                if (r0 + q < m && tt < d) s_x[tt * P + r0 + q] = v[q][h];
            }
        for (int tt = lane + 64; tt < d; tt += 32)   // d > 64: the rest, row by row
            for (int q = 0; q < 4 && r0 + q < m; ++q) s_x[tt * P + r0 + q] = __ldg(X + (int64_t)s_id[r0 + q] * d + tt);
    }
    __syncthreads();
    const int TI = (a + 1) / 2, TJ = (m + 3) / 4;
    for (int tile = threadIdx.x; tile < TI * TJ; tile += kJoinThreads) {
        const int i0 = 2 * (tile / TJ), j0 = 4 * (tile % TJ);
        if (j0 + 3 <= i0) continue;   // no pair j > i in the tile
        float acc[2][4];
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
        for (int tt = 0; tt < d; ++tt) {
            const float *row = s_x + tt * P;
            const float xa0 = row[i0], xa1 = row[i0 + 1];
            float xb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) xb[q] = row[j0 + q];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float u0 = xa0 - xb[q], u1 = xa1 - xb[q];
                acc[0][q] = fmaf(u0, u0, acc[0][q]);
                acc[1][q] = fmaf(u1, u1, acc[1][q]);
            }
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i = i0 + p;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + q;
                if (i >= a || j >= m || j <= i) continue;
                const uint32_t ia = (uint32_t)s_id[i], ib = (uint32_t)s_id[j];
                const unsigned long long ka = make_key(acc[p][q], ib), kb = make_key(acc[p][q], ia);
                // the atomics' results are unused, so they issue as reductions
                // the thread does not wait for
                if (ka < s_thr[i]) atomicMin(cand + (size_t)ia * C + slot_of(ib, lc), ka);
                if (kb < s_thr[j]) atomicMin(cand + (size_t)ib * C + slot_of(ia, lc), kb);
            }
        }
    }
}

// ----------------------------------------------------------------- merge

// Warp per point, points strided over the grid: the list (sorted, k keys)
// and the valid candidates (m distinct keys, none in the list) ranked by
// counting: list entry c goes to c + #candidates below it, candidate q to
// #list keys below it + #candidates below it; ranks under k are kept.
constexpr int kMergeWarps = 8;

__global__ void __launch_bounds__(kMergeWarps * 32)
merge_kernel(int64_t n, int k, int lr, int lc, int t, unsigned long long *__restrict__ ch, long long lim,
             uint64_t *__restrict__ key, unsigned long long *__restrict__ flags,
             unsigned long long *__restrict__ rn, unsigned long long *__restrict__ ro,
             unsigned long long *__restrict__ cand) {
    __shared__ uint64_t s_list[kMergeWarps][kMaxK];
    __shared__ uint64_t s_cand[kMergeWarps][kMaxSlots];
    __shared__ uint64_t s_out[kMergeWarps][kMaxK];
    __shared__ unsigned long long s_cnt[kMergeWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!active(ch, t, lim)) return;   // grid-uniform
    const int R = 1 << lr, C = 1 << lc;
    uint64_t *L = s_list[warp], *Q = s_cand[warp], *O = s_out[warp];
    unsigned long long changed = 0;
    for (int64_t u = (int64_t)blockIdx.x * kMergeWarps + warp; u < n; u += (int64_t)gridDim.x * kMergeWarps) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            if (c < k) L[c] = key[u * k + c];
        }
        for (int s = lane; s < R; s += 32) {
            rn[(size_t)u * R + s] = kEmpty;
            ro[(size_t)u * R + s] = kEmpty;
        }
        __syncwarp();
        int m = 0;
        for (int s0 = 0; s0 < C; s0 += 32) {
            const int s = s0 + lane;
            uint64_t q = kEmpty;
            if (s < C) {
                q = cand[(size_t)u * C + s];
                if (q != kEmpty) cand[(size_t)u * C + s] = kEmpty;
            }
            bool keep = q != kEmpty;
            if (keep) {   // drop a candidate already in the list (same id, same key)
                int lo = 0, hi = k;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (L[mid] < q) lo = mid + 1;
                    else hi = mid;
                }
                keep = !(lo < k && L[lo] == q);
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (keep) Q[m + __popc(b & ((1u << lane) - 1u))] = q;
            m += __popc(b);
        }
        __syncwarp();
        if (m == 0) continue;   // warp-uniform: the list stays as it is
        const unsigned long long fl = flags[u];
        unsigned long long nf = 0;
        int took = 0;
        // list entries
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            if (c < k) {
                const uint64_t x = L[c];
                int r = c;
                for (int i = 0; i < m; ++i) r += Q[i] < x;
                if (r < k) O[r] = x;
            }
        }
        // candidates
        for (int q0 = 0; q0 < m; q0 += 32) {
            const int q = q0 + lane;
            bool kept = false;
            uint64_t x = 0;
            int r = 0;
            if (q < m) {
                x = Q[q];
                int lo = 0, hi = k;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (L[mid] < x) lo = mid + 1;
                    else hi = mid;
                }
                r = lo;
                for (int i = 0; i < m; ++i) r += Q[i] < x;
                kept = r < k;
                if (kept) O[r] = x;
            }
            took += __popc(__ballot_sync(0xffffffffu, kept));
        }
        __syncwarp();
        // new flags by output position: an output key that was in the list
        // keeps its flag, a candidate is new
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            bool isnew = false;
            if (c < k) {
                const uint64_t x = O[c];
                int lo = 0, hi = k;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (L[mid] < x) lo = mid + 1;
                    else hi = mid;
                }
                const bool from_list = lo < k && L[lo] == x;
                isnew = from_list ? ((fl >> lo) & 1ull) != 0 : true;
            }
            nf |= (unsigned long long)__ballot_sync(0xffffffffu, isnew) << (32 * e);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = e * 32 + lane;
            if (c < k) key[u * k + c] = O[c];
        }
        if (lane == 0) flags[u] = nf;
        changed += (unsigned long long)took;
        __syncwarp();
    }
    // one atomic per block
    if (lane == 0) s_cnt[warp] = changed;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < kMergeWarps; ++w) tot += s_cnt[w];
        if (tot) atomicAdd(ch + t, tot);
    }
}

// ---------------------------------------------------------------- output

__global__ void output_kernel(int64_t total, const uint64_t *__restrict__ key, int32_t *__restrict__ idx,
                              float *__restrict__ dist) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint64_t x = key[e];
    idx[e] = (int32_t)(uint32_t)x;
    dist[e] = sqrtf(__uint_as_float((uint32_t)(x >> 32)));
}

}  // namespace nnd

namespace {

struct NndParams {
    int S, R, C, lr, lc, T, P;
    long long lim;
    size_t join_smem;
};

int log2_exact(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return (1 << b) == v ? b : -1;
}

rsc_status nnd_params(int64_t n, int32_t d, int32_t k, const rsc_nnd_opts *o, NndParams *p) {
    if (n < 2 || n >= (int64_t)INT32_MAX) return fail(RSC_ERR_INVALID_ARG, "n = %lld outside [2, 2^31)", (long long)n);
    if (d < 1) return fail(RSC_ERR_INVALID_ARG, "d = %d < 1", d);
    if (k < 2 || k > nnd::kMaxK || k > n) return fail(RSC_ERR_INVALID_ARG, "k = %d outside [2, min(64, n)]", k);
    const rsc_nnd_opts z{};
    const rsc_nnd_opts &q = o ? *o : z;
    p->S = q.sample ? q.sample : k;
    p->R = q.rev_slots ? q.rev_slots : 32;
    p->C = q.cand_slots ? q.cand_slots : 64;
    if (p->S < 1 || p->S > k) return fail(RSC_ERR_INVALID_ARG, "sample = %d outside [1, k]", p->S);
    p->lr = log2_exact(p->R);
    p->lc = log2_exact(p->C);
    if (p->R < 1 || p->R > nnd::kMaxSlots || p->lr < 0)
        return fail(RSC_ERR_INVALID_ARG, "rev_slots = %d is not a power of two in [1, 64]", p->R);
    if (p->C < 1 || p->C > nnd::kMaxSlots || p->lc < 0)
        return fail(RSC_ERR_INVALID_ARG, "cand_slots = %d is not a power of two in [1, 64]", p->C);
    if (q.max_iters < 0 || q.max_iters > nnd::kMaxIters)
        return fail(RSC_ERR_INVALID_ARG, "max_iters = %d outside [0, 64]", q.max_iters);
    p->T = q.max_iters ? q.max_iters : std::max(5, (int)lround(log2((double)n)));
    p->T = std::min(p->T, nnd::kMaxIters);
    if (!(q.delta >= 0.0) || !isfinite(q.delta)) return fail(RSC_ERR_INVALID_ARG, "delta must be finite and >= 0");
    // an iteration with c changes stops the run when c < delta n k, i.e. when
    // c < ceil(delta n k) (c is an integer)
    p->lim = (long long)ceil(q.delta * (double)n * (double)k);
    const int rows = p->S + p->R + k + p->R;   // join rows at most
    p->P = ((rows + 3) / 4) * 4 + 1;           // odd stride, room for 2 x 4 tiles past the last row
    p->join_smem = sizeof(uint64_t) * p->P + sizeof(int32_t) * p->P + sizeof(float) * (size_t)d * p->P;
    if (p->join_smem > 200 * 1024)
        return fail(RSC_ERR_UNSUPPORTED, "d = %d with %d join rows needs %zu bytes of shared memory", d, rows,
                    p->join_smem);
    return RSC_OK;
}

struct NndLayout {
    unsigned int *status;
    uint64_t *key;
    unsigned long long *flags, *smask, *rn, *ro, *cand, *ch, *pairs;
};

NndLayout carve_nnd(void *ws, int64_t n, int k, const NndParams &p, size_t *bytes) {
    Carve cv(ws);
    NndLayout L;
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.ch = cv.take<unsigned long long>(nnd::kMaxIters);
    L.pairs = cv.take<unsigned long long>((size_t)nnd::kMaxIters * nnd::kPairSlots);   // fixed offset: 768 bytes
    L.key = cv.take<uint64_t>((size_t)n * k);
    L.flags = cv.take<unsigned long long>((size_t)n);
    L.smask = cv.take<unsigned long long>((size_t)n);
    L.rn = cv.take<unsigned long long>((size_t)n * p.R);
    L.ro = cv.take<unsigned long long>((size_t)n * p.R);
    L.cand = cv.take<unsigned long long>((size_t)n * p.C);
    if (bytes) *bytes = cv.used;
    return L;
}

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" {

rsc_status rsc_knn_descent_pairs(const void *workspace, size_t workspace_bytes, int64_t *pairs) {
    constexpr size_t off = 768, cnt = (size_t)nnd::kMaxIters * nnd::kPairSlots;
    if (!workspace || !pairs) return fail(RSC_ERR_INVALID_ARG, "workspace or pairs is NULL");
    if (workspace_bytes < off + cnt * sizeof(unsigned long long))
        return fail(RSC_ERR_WORKSPACE, "workspace of %zu bytes holds no counters", workspace_bytes);
    unsigned long long h[cnt];
    RSC_CUDA_TRY(cudaMemcpy(h, static_cast<const char *>(workspace) + off, sizeof h, cudaMemcpyDeviceToHost));
    for (int t = 0; t < nnd::kMaxIters; ++t) {
        unsigned long long s = 0;
        for (int j = 0; j < nnd::kPairSlots; ++j) s += h[t * nnd::kPairSlots + j];
        pairs[t] = (int64_t)s;
    }
    return RSC_OK;
}

rsc_status rsc_knn_descent_workspace_size(int64_t n, int32_t d, int32_t k, const rsc_nnd_opts *opts, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    NndParams p;
    rsc_status s = nnd_params(n, d, k, opts, &p);
    if (s != RSC_OK) return s;
    carve_nnd(nullptr, n, k, p, bytes);
    return RSC_OK;
}

rsc_status rsc_knn_descent(const float *X, int64_t n, int32_t d, int32_t k, const int32_t *init_idx, int32_t *idx,
                           float *dist, int64_t *changes, const rsc_nnd_opts *opts, void *workspace,
                           size_t workspace_bytes) {
    RSC_TRACE("rsc_knn_descent");
    NndParams p;
    rsc_status s = nnd_params(n, d, k, opts, &p);
    if (s != RSC_OK) return s;
    if (!X || !idx || !dist) return fail(RSC_ERR_INVALID_ARG, "X, idx or dist is NULL");
    size_t need = 0;
    carve_nnd(nullptr, n, k, p, &need);
    if (!workspace) return fail(RSC_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(RSC_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, need);
    const NndLayout L = carve_nnd(workspace, n, k, p, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(opts ? opts->stream : nullptr);
    const uint64_t seed = opts ? opts->seed : 0;
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, kStatusBytes, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.ch, 0, sizeof(unsigned long long) * nnd::kMaxIters, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.pairs, 0, sizeof(unsigned long long) * nnd::kMaxIters * nnd::kPairSlots, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.rn, 0xFF, sizeof(unsigned long long) * (size_t)n * p.R, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.ro, 0xFF, sizeof(unsigned long long) * (size_t)n * p.R, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.cand, 0xFF, sizeof(unsigned long long) * (size_t)n * p.C, st));
    nnd::init_kernel<<<(unsigned)ceil_div(n, nnd::kInitWarps), nnd::kInitWarps * 32, 0, st>>>(X, n, d, k, seed,
                                                                                              init_idx, L.key, L.flags);
    RSC_CUDA_TRY(cudaGetLastError());
    if (p.join_smem > 48 * 1024)
        RSC_CUDA_TRY(cudaFuncSetAttribute(nnd::join_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p.join_smem));
    const int merge_grid = (int)std::min<int64_t>(ceil_div(n, nnd::kMergeWarps), (int64_t)sm_count() * 16);
    for (int t = 0; t < p.T; ++t) {
        nnd::sample_kernel<<<(unsigned)ceil_div(n, nnd::kSampleWarps), nnd::kSampleWarps * 32, 0, st>>>(
            n, k, p.S, p.lr, seed, t, L.ch, p.lim, L.key, L.flags, L.smask, L.rn, L.ro);
        nnd::join_kernel<<<(unsigned)n, nnd::kJoinThreads, p.join_smem, st>>>(
            X, n, d, k, p.lr, p.lc, p.P, t, L.ch, p.lim, L.key, L.flags, L.smask, L.rn, L.ro, L.cand, L.pairs);
        nnd::merge_kernel<<<merge_grid, nnd::kMergeWarps * 32, 0, st>>>(n, k, p.lr, p.lc, t, L.ch, p.lim, L.key,
                                                                        L.flags, L.rn, L.ro, L.cand);
        RSC_CUDA_TRY(cudaGetLastError());
    }
    const int64_t total = n * k;
    nnd::output_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(total, L.key, idx, dist);
    RSC_CUDA_TRY(cudaGetLastError());
    if (changes)
        RSC_CUDA_TRY(cudaMemcpyAsync(changes, L.ch, sizeof(int64_t) * nnd::kMaxIters, cudaMemcpyDeviceToDevice, st));
    return RSC_OK;
}

}  // extern "C"
