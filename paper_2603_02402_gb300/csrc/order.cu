// Locality ordering of the rows for the tensor-core candidate search.
//
// The search keeps, per (query row, column part), the best list seen so far
// and admits a tile's values only when one beats the list's threshold.  Rows
// that arrive in random order keep improving the lists for the whole scan
// (about KC * ln(n / KC) improvements per list), and each improvement sends
// the whole warp through the slow insertion path.  When a query first meets
// its own neighbourhood, its thresholds are nearly final after a few tiles
// and the rest of the scan is a pure min-and-compare.
//
// So, before the search, rows are grouped by a two-level k-means:
//   1. C1 coarse centroids start at strided rows; Lloyd iterations run on a
//      strided sample; every row goes to its nearest coarse centroid;
//   2. inside each coarse cluster, C2 sub-centroids (Lloyd on a sample taken
//      in coarse order), and every row goes to the nearest of its cluster's;
//   3. greedy nearest-neighbour chains order the coarse centroids and each
//      cluster's sub-centroids, so neighbouring clusters end up adjacent;
//   4. a stable counting sort by (coarse rank, sub rank) gives perm (sorted
//      position -> original row).
// The search then runs on the permuted operands and each query tile scans
// the database tiles around its own position first.  The ordering changes
// only the order in which candidates are met, never the set of distances
// scanned: the result is still the exact scan's, and the FP32 re-rank maps
// positions back to the original row ids and orders ties by them.
//
// Every step is deterministic: centroid sums run over each cluster's rows in
// row order (after the stable sort) instead of atomics.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace rsc {

namespace {

constexpr int kCentTile = 64;        // centroids staged in shared memory per pass
constexpr int kAssignThreads = 128;
constexpr int kSortWarps = 8;        // warps per block in the counting sort
constexpr int kSub = 1024;           // keys per warp slice
constexpr int kChunk = kSortWarps * kSub;   // keys per block (one count column per chunk)

// Nearest centroid (squared distance |c|^2 - 2 x.c, ties to the lower index)
// of rows i * step, i < m.  Thread per row; DP = padded row length.
template <int DP>
__global__ void __launch_bounds__(kAssignThreads)
assign_kernel(const float *__restrict__ Y, int64_t m, int64_t step, const float *__restrict__ cent,
              const float *__restrict__ cnorm, int C, int32_t *__restrict__ lab) {
    __shared__ __align__(16) float cs[kCentTile][DP];
    __shared__ float cn[kCentTile];
    // two keys per thread (keys i and i + half of the block's span), so every
    // centroid read from shared memory serves both
    const int64_t span = (int64_t)2 * kAssignThreads;
    const int64_t i0 = (int64_t)blockIdx.x * span + threadIdx.x, i1 = i0 + kAssignThreads;
    const bool a0 = i0 < m, a1 = i1 < m;
    float x[DP], z[DP];
    const float4 *xr = reinterpret_cast<const float4 *>(Y + (a0 ? i0 * step : 0) * DP);
    const float4 *zr = reinterpret_cast<const float4 *>(Y + (a1 ? i1 * step : 0) * DP);
#pragma unroll
    for (int t4 = 0; t4 < DP / 4; ++t4) {
        const float4 v = a0 ? xr[t4] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 w = a1 ? zr[t4] : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * t4] = v.x;
        x[4 * t4 + 1] = v.y;
        x[4 * t4 + 2] = v.z;
        x[4 * t4 + 3] = v.w;
        z[4 * t4] = w.x;
        z[4 * t4 + 1] = w.y;
        z[4 * t4 + 2] = w.z;
        z[4 * t4 + 3] = w.w;
    }
    float best0 = INFINITY, best1 = INFINITY;
    int bi0 = 0, bi1 = 0;
    for (int c0 = 0; c0 < C; c0 += kCentTile) {
        const int nc = min(kCentTile, C - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * DP; e += blockDim.x) cs[e / DP][e % DP] = cent[(int64_t)c0 * DP + e];
        for (int e = threadIdx.x; e < nc; e += blockDim.x) cn[e] = cnorm[c0 + e];
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const float4 *cr = reinterpret_cast<const float4 *>(cs[c]);
            float p0 = 0.f, p1 = 0.f, q0 = 0.f, q1 = 0.f;
#pragma unroll
            for (int t4 = 0; t4 < DP / 4; t4 += 2) {
                const float4 u = cr[t4];
                const float4 w = cr[t4 + 1];   // DP is a multiple of 8
                p0 = fmaf(x[4 * t4], u.x, p0);
                p0 = fmaf(x[4 * t4 + 1], u.y, p0);
                p0 = fmaf(x[4 * t4 + 2], u.z, p0);
                p0 = fmaf(x[4 * t4 + 3], u.w, p0);
                p1 = fmaf(x[4 * t4 + 4], w.x, p1);
                p1 = fmaf(x[4 * t4 + 5], w.y, p1);
                p1 = fmaf(x[4 * t4 + 6], w.z, p1);
                p1 = fmaf(x[4 * t4 + 7], w.w, p1);
                q0 = fmaf(z[4 * t4], u.x, q0);
                q0 = fmaf(z[4 * t4 + 1], u.y, q0);
                q0 = fmaf(z[4 * t4 + 2], u.z, q0);
                q0 = fmaf(z[4 * t4 + 3], u.w, q0);
                q1 = fmaf(z[4 * t4 + 4], w.x, q1);
                q1 = fmaf(z[4 * t4 + 5], w.y, q1);
                q1 = fmaf(z[4 * t4 + 6], w.z, q1);
                q1 = fmaf(z[4 * t4 + 7], w.w, q1);
            }
            const float s0 = fmaf(-2.f, p0 + p1, cn[c]), s1 = fmaf(-2.f, q0 + q1, cn[c]);
            if (s0 < best0) {   // strict: the lower index wins ties
                best0 = s0;
                bi0 = c0 + c;
            }
            if (s1 < best1) {
                best1 = s1;
                bi1 = c0 + c;
            }
        }
    }
    if (a0) lab[i0] = bi0;
    if (a1) lab[i1] = bi1;
}
// Centroid c <- row (c * n) / C; its squared norm alongside.
__global__ void init_centroids_kernel(const float *__restrict__ Y, int64_t n, int DP, int C, float *__restrict__ cent,
                                      float *__restrict__ cnorm) {
    const int c = blockIdx.x;
    const int64_t row = ((int64_t)c * n) / C;
    float s = 0.f;
    for (int t = threadIdx.x; t < DP; t += 32) {
        const float v = Y[row * DP + t];
        cent[(int64_t)c * DP + t] = v;
        s = fmaf(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) cnorm[c] = s;
}

// Per-chunk label counts: block b counts keys [b * kChunk, (b + 1) * kChunk)
// into cnt[label * nchunk + b] (kSortWarps warps, shared-memory atomics).
__global__ void __launch_bounds__(kSortWarps * 32)
chunk_hist_kernel(const int32_t *__restrict__ lab, int64_t m, int C, int nchunk, int32_t *__restrict__ cnt) {
    extern __shared__ int32_t hs[];   // [C]
    const int ch = blockIdx.x;
    for (int c = threadIdx.x; c < C; c += blockDim.x) hs[c] = 0;
    __syncthreads();
    const int64_t b = (int64_t)ch * kChunk, e = min(m, b + kChunk);
    for (int64_t r = b + threadIdx.x; r < e; r += blockDim.x) atomicAdd(&hs[lab[r]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) cnt[(int64_t)c * nchunk + ch] = hs[c];
}

// Stable scatter, block per chunk: warp w walks its kSub-key slice of the
// chunk in key order, 32 keys a step; keys with equal labels within a step
// are ranked by lane (match_any) and a per-(warp, label) cursor carries the
// count across steps.  The cursors start at the chunk's offset plus the
// slice histograms of the lower warps.  out[pos] = the row of key r:
// rows[r * step] (rows given) or r * step.
__global__ void __launch_bounds__(kSortWarps * 32)
chunk_scatter_kernel(const int32_t *__restrict__ lab, int64_t m, int64_t step, const int32_t *__restrict__ rows,
                     int C, int nchunk, const int32_t *__restrict__ off, int32_t *__restrict__ out) {
    extern __shared__ int32_t cur_s[];   // [kSortWarps][C]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x;
    int32_t *cur = cur_s + warp * C;
    for (int c = lane; c < C; c += 32) cur[c] = 0;
    __syncwarp();
    const int64_t b = (int64_t)ch * kChunk + (int64_t)warp * kSub, e = min(m, b + kSub);
    for (int64_t r = b + lane; r < e; r += 32) atomicAdd(&cur[lab[r]], 1);
    __syncthreads();
    // exclusive prefix over the warps, per label, plus the chunk offset
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int run = off[(int64_t)c * nchunk + ch];
        for (int w = 0; w < kSortWarps; ++w) {
            const int h = cur_s[w * C + c];
            cur_s[w * C + c] = run;
            run += h;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t r0 = b; r0 < e; r0 += 32) {
        const int64_t r = r0 + lane;
        const bool act = r < e;
        const int c = act ? lab[r] : -1 - lane;   // inactive lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (act) {
            const int pos = cur[c] + __popc(peers & lt);
            out[pos] = rows ? rows[r * step] : (int32_t)(r * step);
        }
        __syncwarp();
        if (act && (peers & lt) == 0) cur[c] += __popc(peers);   // the lowest lane of each label advances it
        __syncwarp();
    }
}

// Centroid c <- mean of its rows (sorted positions [off[c * nchunk],
// off[(c + 1) * nchunk])), summed in row order; an empty cluster keeps its
// centroid.  Warp per centroid.
__global__ void centroid_mean_kernel(const float *__restrict__ Y, int DP, const int32_t *__restrict__ sorted_rows,
                                     const int32_t *__restrict__ off, int nchunk, int C, float *__restrict__ cent,
                                     float *__restrict__ cnorm) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= C) return;
    const int32_t b = off[(int64_t)c * nchunk], e = off[(int64_t)(c + 1) * nchunk];
    if (e == b) return;
    float s0 = 0.f, s1 = 0.f;
    // rows fetched kMeanAhead at a time (independent loads), added in order
    constexpr int kMeanAhead = 8;
    for (int32_t p0 = b; p0 < e; p0 += kMeanAhead) {
        float v0[kMeanAhead], v1[kMeanAhead];
#pragma unroll
        for (int u = 0; u < kMeanAhead; ++u) {
            v0[u] = v1[u] = 0.f;
            if (p0 + u < e) {
                const float *y = Y + (int64_t)sorted_rows[p0 + u] * DP;
                if (lane < DP) v0[u] = y[lane];
                if (lane + 32 < DP) v1[u] = y[lane + 32];
            }
        }
#pragma unroll
        for (int u = 0; u < kMeanAhead; ++u) {
            if (p0 + u < e) {
                s0 += v0[u];
                s1 += v1[u];
            }
        }
    }
    const float inv = 1.f / (float)(e - b);
    s0 *= inv;
    s1 *= inv;
    if (lane < DP) cent[(int64_t)c * DP + lane] = s0;
    if (lane + 32 < DP) cent[(int64_t)c * DP + lane + 32] = s1;
    float q = (lane < DP ? s0 * s0 : 0.f) + (lane + 32 < DP ? s1 * s1 : 0.f);
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) cnorm[c] = q;
}

// Sub-cluster assignment: key i is row rows[i * step] (rows given) or
// i * step; its coarse cluster c1 = lab1[row]; label = c1 * C2 + the nearest
// of c1's C2 sub-centroids (|c|^2 - 2 x.c, ties to the lower index), written
// at out[row] (by_row) or out[i].  Thread per key; the C2 sub-centroids of a
// coarse cluster are read through L1 (neighbouring keys share them).
template <int DP>
__global__ void __launch_bounds__(kAssignThreads)
assign_sub_kernel(const float *__restrict__ Y, int64_t m, int64_t step, const int32_t *__restrict__ rows,
                  const int32_t *__restrict__ lab1, const float *__restrict__ cent2, const float *__restrict__ cnorm2,
                  int C2, bool by_row, const int32_t *__restrict__ rank1, const int32_t *__restrict__ rank2,
                  int32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t row = rows ? (int64_t)rows[i * step] : i * step;
    float x[DP];
    const float4 *xr = reinterpret_cast<const float4 *>(Y + row * DP);
#pragma unroll
    for (int t4 = 0; t4 < DP / 4; ++t4) {
        const float4 v = xr[t4];
        x[4 * t4] = v.x;
        x[4 * t4 + 1] = v.y;
        x[4 * t4 + 2] = v.z;
        x[4 * t4 + 3] = v.w;
    }
    const int base = lab1[row] * C2;
    float best = INFINITY;
    int bi = 0;
    for (int c = 0; c < C2; ++c) {
        const float4 *cr = reinterpret_cast<const float4 *>(cent2 + (int64_t)(base + c) * DP);
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < DP / 4; t4 += 2) {
            const float4 u = __ldg(cr + t4), w = __ldg(cr + t4 + 1);
            a0 = fmaf(x[4 * t4], u.x, a0);
            a0 = fmaf(x[4 * t4 + 1], u.y, a0);
            a0 = fmaf(x[4 * t4 + 2], u.z, a0);
            a0 = fmaf(x[4 * t4 + 3], u.w, a0);
            a1 = fmaf(x[4 * t4 + 4], w.x, a1);
            a1 = fmaf(x[4 * t4 + 5], w.y, a1);
            a1 = fmaf(x[4 * t4 + 6], w.z, a1);
            a1 = fmaf(x[4 * t4 + 7], w.w, a1);
        }
        const float sv = fmaf(-2.f, a0 + a1, cnorm2[base + c]);
        if (sv < best) {
            best = sv;
            bi = c;
        }
    }
    // ranked key (position of the coarse cluster, then of the sub-cluster,
    // along their chains) for the final order; the plain label otherwise
    out[by_row ? row : i] = rank1 ? rank1[base / C2] * C2 + rank2[base + bi] : base + bi;
}

// Sub-centroid s of coarse cluster c <- the row at position b + (s * size) /
// C2 of the cluster's segment [b, b + size) of perm1 (the coarse centroid
// when the cluster is empty).  Warp per sub-centroid.
__global__ void init_sub_centroids_kernel(const float *__restrict__ Y, int DP, const int32_t *__restrict__ perm1,
                                          const int32_t *__restrict__ off1, int nchunk1, int C2,
                                          const float *__restrict__ cent1, float *__restrict__ cent2,
                                          float *__restrict__ cnorm2) {
    const int g = blockIdx.x, c = g / C2, sidx = g % C2;
    const int32_t b = off1[(int64_t)c * nchunk1], e = off1[(int64_t)(c + 1) * nchunk1];
    const float *src = (e > b) ? Y + (int64_t)perm1[b + ((int64_t)sidx * (e - b)) / C2] * DP : cent1 + (int64_t)c * DP;
    float q = 0.f;
    for (int t = threadIdx.x; t < DP; t += 32) {
        const float v = src[t];
        cent2[(int64_t)g * DP + t] = v;
        q = fmaf(v, v, q);
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (threadIdx.x == 0) cnorm2[g] = q;
}

// Greedy nearest-neighbour chain through each group of gsize consecutive
// centroids (cent [groups * gsize, DP]), starting at the group's first:
// rank[c] = position of centroid c along its group's chain (ties to the lower
// index).  Consecutive clusters in the final order are then near each other,
// so tiles that straddle a cluster boundary stay compact.  Block per group,
// gsize <= kChainMax: the block first fills the group's squared-distance
// matrix (every entry summed over t in order), then one warp walks it.
constexpr int kChainMax = 128;
constexpr int kChainThreads = 256;
static_assert(kOrderMaxCoarse <= kChainMax && kOrderSub <= kChainMax, "chain groups fit the seen flags");
__global__ void __launch_bounds__(kChainThreads) chain_kernel(const float *__restrict__ cent, int DP, int gsize,
                                                              int32_t *__restrict__ rank) {
    extern __shared__ float cs[];   // [gsize][DP + 1] (padded against bank conflicts), then [gsize][gsize]
    __shared__ bool seen[kChainMax];
    const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int W = DP + 1;
    float *D = cs + gsize * W;
    const float *C = cent + (int64_t)g * gsize * DP;
    for (int e = tid; e < gsize * DP; e += kChainThreads) cs[(e / DP) * W + e % DP] = C[e];
    for (int c = tid; c < gsize; c += kChainThreads) seen[c] = false;
    __syncthreads();
    for (int e = tid; e < gsize * gsize; e += kChainThreads) {
        const int a = e / gsize, c = e - a * gsize;   // D[a][c] = |cent_c - cent_a|^2
        const float *ca = cs + a * W, *cc = cs + c * W;
        float s = 0.f;
        for (int t = 0; t < DP; ++t) {
            const float df = cc[t] - ca[t];
            s = fmaf(df, df, s);
        }
        D[e] = s;
    }
    __syncthreads();
    if (tid >= 32) return;
    int last = 0;
    if (lane == 0) {
        seen[0] = true;
        rank[(int64_t)g * gsize] = 0;
    }
    __syncwarp();
    for (int pos = 1; pos < gsize; ++pos) {
        float best = INFINITY;
        int bi = INT_MAX;
        const float *dl = D + last * gsize;
        for (int c = lane; c < gsize; c += 32) {
            if (seen[c]) continue;
            const float s = dl[c];
            if (s < best) {
                best = s;
                bi = c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        last = bi;
        if (lane == 0) {
            seen[bi] = true;
            rank[(int64_t)g * gsize + bi] = pos;
        }
        __syncwarp();
    }
}

cudaError_t launch_assign_sub(const float *Y, int DP, int64_t m, int64_t step, const int32_t *rows,
                              const int32_t *lab1, const float *cent2, const float *cnorm2, int C2, bool by_row,
                              const int32_t *rank1, const int32_t *rank2, int32_t *out, cudaStream_t st) {
    const unsigned blocks = (unsigned)ceil_div(m, kAssignThreads);
#define RSC_ASSIGN(dp)                                                                                       \
    case dp:                                                                                                 \
        assign_sub_kernel<dp><<<blocks, kAssignThreads, 0, st>>>(Y, m, step, rows, lab1, cent2, cnorm2, C2, \
                                                                 by_row, rank1, rank2, out);                 \
        break
    switch (DP) {
        RSC_ASSIGN(8);
        RSC_ASSIGN(16);
        RSC_ASSIGN(24);
        RSC_ASSIGN(32);
        RSC_ASSIGN(40);
        RSC_ASSIGN(48);
        RSC_ASSIGN(56);
        RSC_ASSIGN(64);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_ASSIGN
    return cudaGetLastError();
}

cudaError_t launch_assign(const float *Y, int DP, int64_t m, int64_t step, const float *cent, const float *cnorm,
                          int C, int32_t *lab, cudaStream_t st) {
    const unsigned blocks = (unsigned)ceil_div(m, 2 * kAssignThreads);   // two keys per thread
#define RSC_ASSIGN(dp) \
    case dp: assign_kernel<dp><<<blocks, kAssignThreads, 0, st>>>(Y, m, step, cent, cnorm, C, lab); break
    switch (DP) {
        RSC_ASSIGN(8);
        RSC_ASSIGN(16);
        RSC_ASSIGN(24);
        RSC_ASSIGN(32);
        RSC_ASSIGN(40);
        RSC_ASSIGN(48);
        RSC_ASSIGN(56);
        RSC_ASSIGN(64);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_ASSIGN
    return cudaGetLastError();
}

// Stable counting sort of labels lab[0 .. m) -> out (positions hold the row
// of each key: rows[r * step] when rows is given, else r * step).
cudaError_t counting_sort(const int32_t *lab, int64_t m, int64_t step, const int32_t *rows, int C, int32_t *cnt,
                          int32_t *off, int64_t *ssum, int32_t *out, cudaStream_t st) {
    const int nchunk = (int)ceil_div(m, kChunk);
    const size_t sm = sizeof(int32_t) * kSortWarps * C;
    cudaError_t e = cudaFuncSetAttribute(chunk_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(int32_t) * kSortWarps * kOrderMaxLeaves));
    if (e != cudaSuccess) return e;
    chunk_hist_kernel<<<nchunk, kSortWarps * 32, sizeof(int32_t) * C, st>>>(lab, m, C, nchunk, cnt);
    if ((e = seg_scan::launch(cnt, (int64_t)C * nchunk, off, ssum, st)) != cudaSuccess) return e;
    chunk_scatter_kernel<<<nchunk, kSortWarps * 32, sm, st>>>(lab, m, step, rows, C, nchunk, off, out);
    return cudaGetLastError();
}

}  // namespace

OrderShape order_shape(int64_t n) {
    OrderShape s;
    s.C2 = kOrderSub;
    s.C1 = (int)std::min<int64_t>(kOrderMaxCoarse, std::max<int64_t>(1, ceil_div(n, (int64_t)kOrderSub * kOrderLeafRows)));
    s.m1 = std::min<int64_t>(n, (int64_t)s.C1 * 64);
    s.step1 = n / s.m1;
    s.m1 = n / s.step1;                    // keys i * step1, i < m1, all inside [0, n)
    s.m2 = std::min<int64_t>(n, (int64_t)s.C1 * s.C2 * 32);
    s.step2 = n / s.m2;
    s.m2 = n / s.step2;
    s.nchunk = (int)ceil_div(n, kChunk);   // the full sorts have the most chunks
    return s;
}

namespace {

struct OrderLayout {
    float *cent1, *cnorm1, *cent2, *cnorm2;
    int32_t *lab1, *lab, *perm1, *cnt, *off, *srows, *rank1, *rank2;
    int64_t *ssum;
};

OrderLayout order_layout(void *scratch, int64_t n, int DP, const OrderShape &s, int groups, size_t *bytes) {
    Carve cv(scratch);
    OrderLayout L;
    const int C = std::max(s.C1 * s.C2, groups);   // widest counting sort
    L.cent1 = cv.take<float>((size_t)s.C1 * DP);
    L.cnorm1 = cv.take<float>((size_t)s.C1);
    L.cent2 = cv.take<float>((size_t)s.C1 * s.C2 * DP);
    L.cnorm2 = cv.take<float>((size_t)s.C1 * s.C2);
    L.lab1 = cv.take<int32_t>((size_t)n);
    L.lab = cv.take<int32_t>((size_t)n);
    L.perm1 = cv.take<int32_t>((size_t)n);
    const size_t ncnt = (size_t)C * s.nchunk;
    L.cnt = cv.take<int32_t>(ncnt);
    L.off = cv.take<int32_t>(ncnt + 1);
    L.ssum = cv.take<int64_t>(seg_scan::kMaxSegs);
    L.srows = cv.take<int32_t>((size_t)std::max(s.m1, s.m2));
    L.rank1 = cv.take<int32_t>((size_t)s.C1);
    L.rank2 = cv.take<int32_t>((size_t)s.C1 * s.C2);
    if (bytes) *bytes = cv.used;
    return L;
}

}  // namespace

size_t order_scratch_bytes(int64_t n, int DP, int groups) {
    size_t bytes = 0;
    order_layout(nullptr, n, DP, order_shape(n), groups, &bytes);
    return bytes;
}

namespace {

// key[pos] = the group (sample) of row rows[pos]: goff[g] <= row < goff[g + 1].
__global__ void group_key_kernel(const int32_t *__restrict__ rows, int64_t n, const int64_t *__restrict__ goff,
                                 int G, int32_t *__restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (goff[mid] <= r) lo = mid;
        else hi = mid;
    }
    key[i] = lo;
}

}  // namespace

cudaError_t launch_locality_order(const float *Y, int64_t n, int DP, int iters, int32_t *perm, void *scratch,
                                  cudaStream_t st, const int64_t *goff, int G) {
    const OrderShape s = order_shape(n);
    if (DP % 8 != 0 || DP > 64) return cudaErrorInvalidValue;
    if (goff && (G < 1 || G > kOrderMaxLeaves)) return cudaErrorInvalidValue;
    const OrderLayout L = order_layout(scratch, n, DP, s, goff ? G : 0, nullptr);
    const int C = s.C1 * s.C2;
    const int mean_warps = 4;
    cudaError_t e;
    // level 1: coarse k-means (Lloyd on a strided sample), then every row
    init_centroids_kernel<<<s.C1, 32, 0, st>>>(Y, n, DP, s.C1, L.cent1, L.cnorm1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nch1 = (int)ceil_div(s.m1, kChunk);
    for (int it = 0; it < iters; ++it) {
        if ((e = launch_assign(Y, DP, s.m1, s.step1, L.cent1, L.cnorm1, s.C1, L.lab1, st)) != cudaSuccess) return e;
        if ((e = counting_sort(L.lab1, s.m1, s.step1, nullptr, s.C1, L.cnt, L.off, L.ssum, L.srows, st)) != cudaSuccess)
            return e;
        centroid_mean_kernel<<<(unsigned)ceil_div(s.C1, mean_warps), mean_warps * 32, 0, st>>>(
            Y, DP, L.srows, L.off, nch1, s.C1, L.cent1, L.cnorm1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_assign(Y, DP, n, 1, L.cent1, L.cnorm1, s.C1, L.lab1, st)) != cudaSuccess) return e;
    if ((e = counting_sort(L.lab1, n, 1, nullptr, s.C1, L.cnt, L.off, L.ssum, L.perm1, st)) != cudaSuccess) return e;
    // level 2: C2 sub-clusters inside each coarse cluster (sample in coarse order)
    init_sub_centroids_kernel<<<C, 32, 0, st>>>(Y, DP, L.perm1, L.off, s.nchunk, s.C2, L.cent1, L.cent2, L.cnorm2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nch2 = (int)ceil_div(s.m2, kChunk);
    for (int it = 0; it < iters; ++it) {
        if ((e = launch_assign_sub(Y, DP, s.m2, s.step2, L.perm1, L.lab1, L.cent2, L.cnorm2, s.C2, false, nullptr,
                                   nullptr, L.lab, st)) != cudaSuccess)
            return e;
        if ((e = counting_sort(L.lab, s.m2, s.step2, L.perm1, C, L.cnt, L.off, L.ssum, L.srows, st)) != cudaSuccess) return e;
        centroid_mean_kernel<<<(unsigned)ceil_div(C, mean_warps), mean_warps * 32, 0, st>>>(Y, DP, L.srows, L.off,
                                                                                            nch2, C, L.cent2,
                                                                                            L.cnorm2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // chains through the coarse centroids and through each cluster's sub-centroids
    const size_t sm1 = sizeof(float) * s.C1 * (DP + 1 + s.C1), sm2 = sizeof(float) * s.C2 * (DP + 1 + s.C2);
    if ((e = cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max(sm1, sm2))) != cudaSuccess)
        return e;
    chain_kernel<<<1, kChainThreads, sm1, st>>>(L.cent1, DP, s.C1, L.rank1);
    chain_kernel<<<s.C1, kChainThreads, sm2, st>>>(L.cent2, DP, s.C2, L.rank2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // every row (walked in coarse order, so a block shares its sub-centroids), keyed by its ranks; the final sort
    if ((e = launch_assign_sub(Y, DP, n, 1, L.perm1, L.lab1, L.cent2, L.cnorm2, s.C2, true, L.rank1, L.rank2, L.lab,
                               st)) != cudaSuccess)
        return e;
    if (!goff) return counting_sort(L.lab, n, 1, nullptr, C, L.cnt, L.off, L.ssum, perm, st);
    // groups (samples) keep their row ranges: the cluster order, then a stable
    // partition by group (perm1 and lab1 are free again)
    if ((e = counting_sort(L.lab, n, 1, nullptr, C, L.cnt, L.off, L.ssum, L.perm1, st)) != cudaSuccess) return e;
    group_key_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(L.perm1, n, goff, G, L.lab1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return counting_sort(L.lab1, n, 1, L.perm1, G, L.cnt, L.off, L.ssum, perm, st);
}

}  // namespace rsc
