// Learned partitioner for pruned exact-distance kNN (candidate pruning on top
// of the brute-force method; the paper's kNN runs through cuVS and its CPU
// side through PyNNDescent, Methods, "Benchmarking" and "Dimensionality
// reduction and graph analysis").
//
//   parts     1024 k-means cells fitted on a training subsample
//   labels    each training cell's exact k nearest cells (brute force over
//             the whole data set, tensor-core search + exact re-rank) give a
//             soft target: the histogram of those neighbours' cells
//   network   MLP d -> H -> H -> P (ReLU), trained on the GPU with the
//             library's kernels: tcgen05 tensor-core GEMMs (mlp_tc.cu) with
//             bfloat16 operands and FP32 accumulation (a SIMT GEMM in the
//             FP32-weight mode), softmax cross-entropy, Adam
//   index     every database cell goes to the part its network output ranks
//             first; rows are counting-sorted by part
//   search    each query probes the n_probe parts its network ranks highest
//             (or, as the baseline without the network, its n_probe nearest
//             centroids); query rows are gathered per probed part and the
//             tensor-core kernel scans only that part's rows; the probed
//             parts' candidates are re-scored exactly in FP32 and merged.
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "knn_tc.cuh"

struct rsc_partitioner;

namespace rsc {

namespace part {

// ------------------------------------------------------------------- GEMM

constexpr int GM = 64, GN = 64, GK = 16;

enum GemmFlags { kRoundA = 1, kRoundB = 2, kReluA = 4, kReluB = 8 };

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = A[m*sam + k*sak],
// B(k, n) = B[k*sbk + n*sbn].  Operands can be passed through ReLU and/or
// rounded to bfloat16 on load; accumulation is FP32 in a fixed k order.
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const float *__restrict__ A, int64_t sam, int64_t sak, const float *__restrict__ B,
            int64_t sbk, int64_t sbn, float *__restrict__ C, int64_t ldc, const float *__restrict__ bias,
            int flags) {
    __shared__ float As[GK][GM + 1];
    __shared__ float Bs[GK][GN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GM; e += 256) {
            const int k = e / GM, m = e % GM;
            float v = 0.f;
            if (m0 + m < M && k0 + k < K) {
                v = A[(int64_t)(m0 + m) * sam + (int64_t)(k0 + k) * sak];
                if (flags & kReluA) v = fmaxf(v, 0.f);
                if (flags & kRoundA) v = bf16r(v);
            }
            As[k][m] = v;
        }
        for (int e = threadIdx.x; e < GK * GN; e += 256) {
            const int k = e / GN, nn = e % GN;
            float v = 0.f;
            if (n0 + nn < N && k0 + k < K) {
                v = B[(int64_t)(k0 + k) * sbk + (int64_t)(n0 + nn) * sbn];
                if (flags & kReluB) v = fmaxf(v, 0.f);
                if (flags & kRoundB) v = bf16r(v);
            }
            Bs[k][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + tx * 4 + j;
            if (nn >= N) continue;
            C[(int64_t)m * ldc + nn] = acc[i][j] + (bias ? bias[nn] : 0.f);
        }
    }
}

void gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B,
          int64_t sbk, int64_t sbn, float *C, int64_t ldc, const float *bias, int flags) {
    dim3 grid((unsigned)ceil_div(N, GN), (unsigned)ceil_div(M, GM));
    gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags);
}

// ------------------------------------------------- loss and optimiser steps

// Warp per row: loss_row = -sum_p t_p (z_p - lse); dz = (softmax * sum(t) - t) / B.
__global__ void softmax_xent_kernel(int B, int P, const float *__restrict__ Z, const float *__restrict__ T,
                                    float *__restrict__ dZ, float *__restrict__ loss_sum) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const float *z = Z + (int64_t)warp * P;
    const float *t = T + (int64_t)warp * P;
    float zmax = -INFINITY;
    for (int p = lane; p < P; p += 32) zmax = fmaxf(zmax, z[p]);
    for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    float se = 0.f, ts = 0.f, tz = 0.f;
    for (int p = lane; p < P; p += 32) {
        se += expf(z[p] - zmax);
        ts += t[p];
        tz += t[p] * (z[p] - zmax);
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
        tz += __shfl_xor_sync(0xffffffffu, tz, o);
    }
    const float lse = logf(se);   // relative to zmax
    if (dZ) {
        float *dz = dZ + (int64_t)warp * P;
        for (int p = lane; p < P; p += 32) dz[p] = (expf(z[p] - zmax - lse) * ts - t[p]) / (float)B;
    }
    if (lane == 0 && loss_sum) atomicAdd(loss_sum, ts * lse - tz);
}

__global__ void relu_bwd_kernel(int64_t count, const float *__restrict__ dA, const float *__restrict__ Z,
                                float *__restrict__ dZ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dZ[i] = Z[i] > 0.f ? dA[i] : 0.f;
}

__global__ void colsum_kernel(int M, int N, const float *__restrict__ X, float *__restrict__ out) {
    const int nn = blockIdx.x * blockDim.x + threadIdx.x;
    if (nn >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += X[(int64_t)m * N + nn];
    out[nn] = s;
}

__global__ void adam_kernel(int64_t count, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------ data movement

__global__ void gather_rows_kernel(const int32_t *__restrict__ rows, int64_t count, const float *__restrict__ X,
                                   int d, float *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * d) return;
    const int64_t r = e / d;
    out[e] = X[(int64_t)rows[r] * d + (e - r * d)];
}

// Soft targets of batch row b (training position pos[b]):
// T[b, p] = (1/k) #{c : labels[nbr[pos[b], c]] = p}.  T must be zeroed.
__global__ void targets_kernel(int B, int k, const int32_t *__restrict__ pos, const int32_t *__restrict__ nbr,
                               const int32_t *__restrict__ labels, int P, float *__restrict__ T) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * k) return;
    const int64_t b = e / k;
    const int c = (int)(e - b * k);
    const int32_t j = nbr[(int64_t)pos[b] * k + c];
    if (j >= 0) atomicAdd(&T[b * P + labels[j]], 1.f / (float)k);
}

// Copy 128-byte operand rows: dst[i] = src[map[i]].
__global__ void permute_rows_kernel(const uint4 *__restrict__ src, const int32_t *__restrict__ map, int64_t rows,
                                    uint4 *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * 8) return;
    const int64_t r = e >> 3;
    dst[e] = src[(int64_t)map[r] * 8 + (e & 7)];
}

// ------------------------------------------------------- k-means / routing

constexpr int kCentTile = 64;

// Thread per point: the R nearest centroids (squared distance, ties by
// index); R = 1 gives the k-means assignment.
template <int R>
__global__ void __launch_bounds__(128)
nearest_centroids_kernel(const float *__restrict__ X, const int32_t *__restrict__ rows, int64_t npts, int d,
                         const float *__restrict__ Cn, int P, int32_t *__restrict__ out) {
    __shared__ float cs[kCentTile][65];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < npts;
    float x[64];
    const int64_t row = active ? (rows ? rows[i] : i) : 0;
#pragma unroll
    for (int t = 0; t < 64; ++t) x[t] = (active && t < d) ? X[row * d + t] : 0.f;
    float bk[R];
    int bi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        bk[r] = INFINITY;
        bi[r] = INT_MAX;
    }
    for (int c0 = 0; c0 < P; c0 += kCentTile) {
        __syncthreads();
        for (int e = threadIdx.x; e < kCentTile * 64; e += blockDim.x) {
            const int c = e / 64, t = e % 64;
            cs[c][t] = (c0 + c < P && t < d) ? Cn[(int64_t)(c0 + c) * d + t] : 0.f;
        }
        __syncthreads();
        for (int c = 0; c < kCentTile && c0 + c < P; ++c) {
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < 64; ++t) {
                const float diff = x[t] - cs[c][t];
                s = fmaf(diff, diff, s);
            }
            const int id = c0 + c;
            if (s < bk[R - 1] || (s == bk[R - 1] && id < bi[R - 1])) {
                // sorted insertion by (s, id)
                int pos = R - 1;
#pragma unroll
                for (int r = R - 1; r > 0; --r) {
                    const bool after = (s < bk[r - 1]) || (s == bk[r - 1] && id < bi[r - 1]);
                    if (after && pos == r) {
                        bk[r] = bk[r - 1];
                        bi[r] = bi[r - 1];
                        pos = r - 1;
                    }
                }
                bk[pos] = s;
                bi[pos] = id;
            }
        }
    }
    if (active)
#pragma unroll
        for (int r = 0; r < R; ++r) out[i * R + r] = bi[r];
}

__global__ void kmeans_accum_kernel(const float *__restrict__ X, const int32_t *__restrict__ rows, int64_t npts,
                                    int d, const int32_t *__restrict__ lab, float *__restrict__ sums,
                                    int32_t *__restrict__ counts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npts * d) return;
    const int64_t i = e / d;
    const int t = (int)(e - i * d);
    const int c = lab[i];
    atomicAdd(&sums[(int64_t)c * d + t], X[(int64_t)rows[i] * d + t]);
    if (t == 0) atomicAdd(&counts[c], 1);
}

__global__ void kmeans_finalize_kernel(int P, int d, const float *__restrict__ sums, const int32_t *__restrict__ counts,
                                       float *__restrict__ Cn) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * d) return;
    const int c = e / d;
    if (counts[c] > 0) Cn[e] = sums[e] / (float)counts[c];   // empty cluster keeps its centroid
}

// Warp per row of logits: the R largest (ties by index) -> out[row * R + r].
template <int R>
__global__ void top_logits_kernel(int64_t rows, int P, const float *__restrict__ Z, int32_t *__restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows) return;
    const float *z = Z + w * P;
    float bk[R];
    int bi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        bk[r] = -INFINITY;
        bi[r] = INT_MAX;
    }
    // per-lane sorted top-R (descending value, ascending id)
    for (int p = lane; p < P; p += 32) {
        const float v = z[p];
        if (v > bk[R - 1] || (v == bk[R - 1] && p < bi[R - 1])) {
            int pos = R - 1;
#pragma unroll
            for (int r = R - 1; r > 0; --r) {
                const bool after = (v > bk[r - 1]) || (v == bk[r - 1] && p < bi[r - 1]);
                if (after && pos == r) {
                    bk[r] = bk[r - 1];
                    bi[r] = bi[r - 1];
                    pos = r - 1;
                }
            }
            bk[pos] = v;
            bi[pos] = p;
        }
    }
    // merge across lanes: R rounds of a warp-wide arg-max
    for (int r = 0; r < R; ++r) {
        float v = bk[0];
        int id = bi[0];
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, id, o);
            if (ov > v || (ov == v && oi < id)) {
                v = ov;
                id = oi;
            }
        }
        if (lane == 0) out[w * R + r] = id;
        if (bi[0] == id) {   // the owning lane pops its head
#pragma unroll
            for (int s = 0; s < R - 1; ++s) {
                bk[s] = bk[s + 1];
                bi[s] = bi[s + 1];
            }
            bk[R - 1] = -INFINITY;
            bi[R - 1] = INT_MAX;
        }
    }
}

// ----------------------------------------------- counting sort by part

__global__ void histogram_kernel(int64_t count, const int32_t *__restrict__ key, int32_t *__restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) atomicAdd(&hist[key[i]], 1);
}

// Single block: off[0] = 0, off[p + 1] = off[p] + cnt[p] (int64); also item
// offsets ceil(cnt / tile) when items != nullptr.
__global__ void __launch_bounds__(1024)
offsets_kernel(int P, const int32_t *__restrict__ cnt, int64_t *__restrict__ off, int tile,
               int32_t *__restrict__ items) {
    // serial scan over at most 1024 entries by thread 0 (tiny)
    if (threadIdx.x == 0) {
        int64_t a = 0;
        int32_t b = 0;
        for (int p = 0; p < P; ++p) {
            off[p] = a;
            if (items) items[p] = b;
            a += cnt[p];
            if (items) b += (int32_t)((cnt[p] + tile - 1) / tile);
        }
        off[P] = a;
        if (items) items[P] = b;
    }
}

__global__ void scatter_kernel(int64_t count, const int32_t *__restrict__ key, const int64_t *__restrict__ off,
                               int32_t *__restrict__ cursor, int32_t *__restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int k = key[i];
    perm[off[k] + atomicAdd(&cursor[k], 1)] = (int32_t)i;
}

// Probe slots: the (query, probe) pairs grouped by part.  slot = position in
// the grouped order; gq[slot] = query, gpos[query * R + r] = slot.
__global__ void probe_scatter_kernel(int64_t nq, int R, const int32_t *__restrict__ route,
                                     const int64_t *__restrict__ off, int32_t *__restrict__ cursor,
                                     int32_t *__restrict__ gq, int64_t *__restrict__ gpos) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq * R) return;
    const int p = route[e];
    const int64_t slot = off[p] + atomicAdd(&cursor[p], 1);
    gq[slot] = (int32_t)(e / R);
    gpos[e] = slot;
}

__global__ void iota64_kernel(int64_t count, int64_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = i;
}

__global__ void set_segment_kernel(int32_t *__restrict__ cnt, int32_t c0, int64_t *__restrict__ doff, int64_t d0,
                                   int64_t d1) {
    cnt[0] = c0;
    doff[0] = d0;
    doff[1] = d1;
}

__global__ void add_offset_kernel(int64_t count, int32_t *__restrict__ a, int32_t off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] += off;
}

// out[j] = base[pos[j]] (composed row ids).
__global__ void compose_kernel(int64_t count, const int32_t *__restrict__ pos, const int32_t *__restrict__ base,
                               int32_t *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) out[j] = base[pos[j]];
}

// ------------------------------------------------ exact merge re-rank

constexpr int kRWarps = 4;

__device__ __forceinline__ bool pgt(float ka, int ia, float kb, int ib) { return ka > kb || (ka == kb && ia > ib); }

// Warp per query: the R probed slots' candidate lists (ids in the database's
// sorted order, mapped through perm; perm == nullptr: identity) are re-scored
// by direct difference in FP32 over X and the k best by (distance, id) kept.
__global__ void __launch_bounds__(kRWarps * 32)
rerank_probe_kernel(const float *__restrict__ X, int d, const int32_t *__restrict__ qrows, int64_t q_base,
                    int64_t nq, int R,
                    const int64_t *__restrict__ gpos, const int32_t *__restrict__ cand, int per_slot,
                    const int32_t *__restrict__ perm, int64_t n_db, int C2, int k, int32_t *__restrict__ idx,
                    float *__restrict__ dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xq = reinterpret_cast<float *>(smem) + warp * 64;
    float *sk = reinterpret_cast<float *>(smem) + kRWarps * 64 + warp * C2;
    int *si = reinterpret_cast<int *>(reinterpret_cast<float *>(smem) + kRWarps * 64 + kRWarps * C2) + warp * C2;
    const int64_t q = (int64_t)blockIdx.x * kRWarps + warp;
    if (q >= nq) return;
    const int64_t row = qrows ? qrows[q] : q_base + q;
    for (int t = lane; t < d; t += 32) xq[t] = X[row * d + t];
    __syncwarp();
    const int C = R * per_slot;
    for (int c = lane; c < C2; c += 32) {
        float key = INFINITY;
        int id = INT_MAX;
        if (c < C) {
            const int r = c / per_slot;
            const int32_t j = cand[gpos[q * R + r] * per_slot + (c - r * per_slot)];
            if (j >= 0 && (int64_t)j < n_db) {   // ids outside [0, n_db) (an aborted search) are skipped
                const int32_t o = perm ? perm[j] : j;
                const float *yr = X + (int64_t)o * d;
                float acc = 0.f;
                for (int t = 0; t < d; ++t) {
                    const float diff = xq[t] - __ldg(yr + t);
                    acc = fmaf(diff, diff, acc);
                }
                key = acc;
                id = o;
            }
        }
        sk[c] = key;
        si[c] = id;
    }
    __syncwarp();
    for (int size = 2; size <= C2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < C2 / 2; i += 32) {
                const int a = (i / stride) * 2 * stride + (i % stride), b = a + stride;
                const bool asc = (a & size) == 0;
                const float ka = sk[a], kb = sk[b];
                const int ia = si[a], ib = si[b];
                if (asc ? pgt(ka, ia, kb, ib) : pgt(kb, ib, ka, ia)) {
                    sk[a] = kb;
                    sk[b] = ka;
                    si[a] = ib;
                    si[b] = ia;
                }
            }
            __syncwarp();
        }
    }
    for (int c = lane; c < k; c += 32) {
        const bool valid = si[c] != INT_MAX;
        idx[q * k + c] = valid ? si[c] : -1;
        dist[q * k + c] = valid ? sqrtf(sk[c]) : INFINITY;
    }
}

}  // namespace part

// ----------------------------------------------------- probe work policy

namespace tck {

// Segments of gathered query rows scanned against database row ranges:
// segment p = query slots [goff[p], goff[p+1]) x database rows [doff[p], doff[p+1]).
struct ProbeWork {
    static constexpr int kShort = 0;
    static constexpr bool kResume = false;
    static constexpr bool kHitHeavy = false;
    static constexpr bool kStartBelow = false;
    static constexpr bool kDynamic = true;   // segments differ in size
    int P;
    const int64_t *goff;
    const int64_t *doff;
    const int32_t *item_off;   // [P + 1] first work item of each segment
    int32_t *cand;             // [slots, EG * KCP]
    int *counter;              // next item (zeroed before the launch)

    int64_t count_host() const { return INT_MAX; }   // the grid is sized by the SM count
    __device__ __forceinline__ int count() const { return item_off[P]; }
    __device__ __forceinline__ WorkItem get(int it) const {
        int lo = 0, hi = P;   // item_off[lo] <= it < item_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (item_off[mid] <= it) lo = mid;
            else hi = mid;
        }
        WorkItem w;
        w.q0 = goff[lo] + (int64_t)(it - item_off[lo]) * BM;
        w.q_end = min(goff[lo + 1], w.q0 + BM);
        w.j_begin = doff[lo];
        w.j_end = doff[lo + 1];
        w.tag = lo;
        w.short_list = false;
        w.win_lo = w.win_hi = w.win_c = 0;
        w.tiles = nullptr;
        w.n_tiles = 0;
        w.skip_window = false;
        return w;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &, int part, int64_t q, const RowTopK<KCP> &list) const {
        int32_t *out = cand + (q * EG + part) * KCP;
#pragma unroll
        for (int c = 0; c < KCP; ++c) out[c] = list.id[c];
    }
};

}  // namespace tck
}  // namespace rsc

// ===================================================================== handle

using namespace rsc;

struct rsc_partitioner {
    int d = 0, P = 0, H = 0, bf16 = 1;
    uint64_t seed = 0;
    int64_t np = 0;           // parameter count
    float *params = nullptr;  // [W1, b1, W2, b2, W3, b3] FP32 master copy
    float *adam_m = nullptr, *adam_v = nullptr;
    int64_t step = 0;
    float *centroids = nullptr;   // [P, d]
    // index over a database
    int64_t n_db = 0;
    int32_t *perm = nullptr;      // sorted position -> row
    int64_t *doff = nullptr;      // [P + 1]
    void *Db_sorted = nullptr;    // [n_db, 64] bf16 operand rows in part order
    unsigned int *status = nullptr;   // device word: failures of the training kernels
};

namespace {

constexpr int kSlotList = 16;     // ids per (slot, column part)
constexpr int kSlotParts = 4;     // column parts per slot (k <= 16)
constexpr int kPerSlot = kSlotList * kSlotParts;
constexpr int kChunkRows = 32768; // network rows per forward chunk
constexpr int kMaxProbe = 8;

int64_t w1_off(const rsc_partitioner *) { return 0; }
int64_t b1_off(const rsc_partitioner *p) { return (int64_t)p->H * p->d; }
int64_t w2_off(const rsc_partitioner *p) { return b1_off(p) + p->H; }
int64_t b2_off(const rsc_partitioner *p) { return w2_off(p) + (int64_t)p->H * p->H; }
int64_t w3_off(const rsc_partitioner *p) { return b2_off(p) + p->H; }
int64_t b3_off(const rsc_partitioner *p) { return w3_off(p) + (int64_t)p->P * p->H; }

// One GEMM of the network: on the tensor cores with BF16 operands (both
// rounded) when the handle uses BF16 weights, else the FP32 SIMT GEMM
// (`flags` then says which operands it rounds).
void mgemm(const rsc_partitioner *p, cudaStream_t st, unsigned int *status, int M, int N, int K, const float *A,
           int64_t sam, int64_t sak, const float *B, int64_t sbk, int64_t sbn, float *C, int64_t ldc,
           const float *bias, int flags) {
    if (p->bf16)
        launch_tc_gemm(st, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags & (part::kReluA | part::kReluB),
                       status);
    else
        part::gemm(st, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags);
}

// Forward of B rows (FP32 [B, d] in Xb): Z1, Z2 [B, H], Z3 [B, P] pre-activations.
void mlp_forward(const rsc_partitioner *p, cudaStream_t st, int B, const float *Xb, float *Z1, float *Z2, float *Z3,
                 unsigned int *status) {
    const int r = p->bf16 ? (part::kRoundA | part::kRoundB) : 0;
    const float *W = p->params;
    mgemm(p, st, status, B, p->H, p->d, Xb, p->d, 1, W + w1_off(p), 1, p->d, Z1, p->H, W + b1_off(p), r);
    mgemm(p, st, status, B, p->H, p->H, Z1, p->H, 1, W + w2_off(p), 1, p->H, Z2, p->H, W + b2_off(p),
          r | part::kReluA);
    mgemm(p, st, status, B, p->P, p->H, Z2, p->H, 1, W + w3_off(p), 1, p->H, Z3, p->P, W + b3_off(p),
          r | part::kReluA);
}

struct TrainBufs {
    float *Xb, *T, *Z1, *Z2, *Z3, *dZ3, *dA, *dZ, *grad, *loss;
};

// Loss (summed into *loss) and gradient of a batch; grad fully overwritten.
void mlp_loss_grad(const rsc_partitioner *p, cudaStream_t st, int B, const TrainBufs &b) {
    const int rw = p->bf16 ? part::kRoundB : 0;   // weights as the B operand
    const int ra = p->bf16 ? part::kRoundB : 0;   // activations as the B operand of dW
    const float *W = p->params;
    float *g = b.grad;
    mlp_forward(p, st, B, b.Xb, b.Z1, b.Z2, b.Z3, p->status);
    part::softmax_xent_kernel<<<(unsigned)ceil_div((int64_t)B * 32, 256), 256, 0, st>>>(B, p->P, b.Z3, b.T, b.dZ3,
                                                                                          b.loss);
    const int H = p->H, P = p->P, d = p->d;
    // layer 3: dW3 = dZ3^T relu(Z2); db3 = colsum(dZ3); dA2 = dZ3 W3
    mgemm(p, st, p->status, P, H, B, b.dZ3, 1, P, b.Z2, H, 1, g + w3_off(p), H, nullptr, ra | part::kReluB);
    part::colsum_kernel<<<(unsigned)ceil_div(P, 256), 256, 0, st>>>(B, P, b.dZ3, g + b3_off(p));
    mgemm(p, st, p->status, B, H, P, b.dZ3, P, 1, W + w3_off(p), H, 1, b.dA, H, nullptr, rw);
    part::relu_bwd_kernel<<<(unsigned)ceil_div((int64_t)B * H, 256), 256, 0, st>>>((int64_t)B * H, b.dA, b.Z2, b.dZ);
    // layer 2
    mgemm(p, st, p->status, H, H, B, b.dZ, 1, H, b.Z1, H, 1, g + w2_off(p), H, nullptr, ra | part::kReluB);
    part::colsum_kernel<<<(unsigned)ceil_div(H, 256), 256, 0, st>>>(B, H, b.dZ, g + b2_off(p));
    mgemm(p, st, p->status, B, H, H, b.dZ, H, 1, W + w2_off(p), H, 1, b.dA, H, nullptr, rw);
    part::relu_bwd_kernel<<<(unsigned)ceil_div((int64_t)B * H, 256), 256, 0, st>>>((int64_t)B * H, b.dA, b.Z1, b.dZ);
    // layer 1: dW1 = dZ1^T x
    mgemm(p, st, p->status, H, d, B, b.dZ, 1, H, b.Xb, d, 1, g + w1_off(p), d, nullptr, ra);
    part::colsum_kernel<<<(unsigned)ceil_div(H, 256), 256, 0, st>>>(B, H, b.dZ, g + b1_off(p));
}

// Failure recorded by the handle's training kernels (read and cleared; the
// stream has been synchronised).
rsc_status take_status(const rsc_partitioner *p, cudaStream_t st) {
    unsigned int word = 0;
    RSC_CUDA_TRY(cudaMemcpyAsync(&word, p->status, sizeof(word), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(word), st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    if (word != 0) return fail((rsc_status)word, "a training kernel recorded status %u", word);
    return RSC_OK;
}

rsc_status check_handle(const rsc_partitioner *p) {
    if (!p || !p->params) return fail(RSC_ERR_INVALID_ARG, "partitioner handle is NULL or destroyed");
    return RSC_OK;
}

}  // namespace

extern "C" {

rsc_status rsc_partitioner_create(int32_t d, int32_t n_parts, int32_t hidden, int32_t bf16_weights, uint64_t seed,
                                  rsc_partitioner **out) {
    if (!out) return fail(RSC_ERR_INVALID_ARG, "out is NULL");
    if (d < 1 || d > 61) return fail(RSC_ERR_INVALID_ARG, "d=%d out of [1, 61]", d);
    if (n_parts < 8 || n_parts > 1024) return fail(RSC_ERR_INVALID_ARG, "n_parts=%d out of [8, 1024]", n_parts);
    if (hidden < 8 || hidden > 1024) return fail(RSC_ERR_INVALID_ARG, "hidden=%d out of [8, 1024]", hidden);
    rsc_partitioner *p = new rsc_partitioner();
    p->d = d;
    p->P = n_parts;
    p->H = hidden;
    p->bf16 = bf16_weights ? 1 : 0;
    p->seed = seed;
    p->np = (int64_t)hidden * d + hidden + (int64_t)hidden * hidden + hidden + (int64_t)n_parts * hidden + n_parts;
    // He-normal initial weights (seeded), zero biases
    std::vector<float> h(p->np, 0.f);
    std::mt19937_64 gen(seed);
    auto fill = [&](int64_t off, int64_t rows, int64_t cols, double scale) {
        std::normal_distribution<double> nd(0.0, scale);
        for (int64_t i = 0; i < rows * cols; ++i) h[off + i] = (float)nd(gen);
    };
    fill(w1_off(p), hidden, d, sqrt(2.0 / d));
    fill(w2_off(p), hidden, hidden, sqrt(2.0 / hidden));
    fill(w3_off(p), n_parts, hidden, sqrt(1.0 / hidden));
    cudaError_t e = cudaMalloc(&p->params, sizeof(float) * p->np);
    if (e == cudaSuccess) e = cudaMalloc(&p->adam_m, sizeof(float) * p->np);
    if (e == cudaSuccess) e = cudaMalloc(&p->adam_v, sizeof(float) * p->np);
    if (e == cudaSuccess) e = cudaMalloc(&p->centroids, sizeof(float) * (size_t)n_parts * d);
    if (e == cudaSuccess) e = cudaMalloc(&p->status, kStatusBytes);
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, kStatusBytes);
    if (e == cudaSuccess) e = cudaMemcpy(p->params, h.data(), sizeof(float) * p->np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->adam_m, 0, sizeof(float) * p->np);
    if (e == cudaSuccess) e = cudaMemset(p->adam_v, 0, sizeof(float) * p->np);
    if (e == cudaSuccess) e = cudaMemset(p->centroids, 0, sizeof(float) * (size_t)n_parts * d);
    if (e != cudaSuccess) {
        cudaFree(p->params);
        cudaFree(p->adam_m);
        cudaFree(p->adam_v);
        cudaFree(p->centroids);
        cudaFree(p->status);
        delete p;
        return fail(RSC_ERR_CUDA, "partitioner allocation failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return RSC_OK;
}

rsc_status rsc_partitioner_destroy(rsc_partitioner *p) {
    if (!p) return RSC_OK;
    cudaFree(p->params);
    cudaFree(p->adam_m);
    cudaFree(p->adam_v);
    cudaFree(p->centroids);
    cudaFree(p->status);
    cudaFree(p->perm);
    cudaFree(p->doff);
    cudaFree(p->Db_sorted);
    delete p;
    return RSC_OK;
}

rsc_status rsc_partitioner_param_count(const rsc_partitioner *p, int64_t *count) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!count) return fail(RSC_ERR_INVALID_ARG, "count is NULL");
    *count = p->np;
    return RSC_OK;
}

rsc_status rsc_partitioner_get_params(const rsc_partitioner *p, float *host_out) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!host_out) return fail(RSC_ERR_INVALID_ARG, "host_out is NULL");
    RSC_CUDA_TRY(cudaMemcpy(host_out, p->params, sizeof(float) * p->np, cudaMemcpyDeviceToHost));
    return RSC_OK;
}

rsc_status rsc_partitioner_set_params(rsc_partitioner *p, const float *host_in) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!host_in) return fail(RSC_ERR_INVALID_ARG, "host_in is NULL");
    RSC_CUDA_TRY(cudaMemcpy(p->params, host_in, sizeof(float) * p->np, cudaMemcpyHostToDevice));
    RSC_CUDA_TRY(cudaMemset(p->adam_m, 0, sizeof(float) * p->np));
    RSC_CUDA_TRY(cudaMemset(p->adam_v, 0, sizeof(float) * p->np));
    p->step = 0;
    return RSC_OK;
}

rsc_status rsc_partitioner_loss_grad_workspace_size(const rsc_partitioner *p, int32_t batch, size_t *bytes) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!bytes || batch < 1) return fail(RSC_ERR_INVALID_ARG, "bytes / batch");
    const size_t B = batch;
    *bytes = kStatusBytes + 256 * 8 +
             sizeof(float) * (B * p->H * 4 + B * p->P * 2 + p->np + 64);
    return RSC_OK;
}

rsc_status rsc_partitioner_loss_grad(rsc_partitioner *p, const float *Xb, const float *T, int32_t batch,
                                     float *loss_host, float *grad, void *workspace, size_t workspace_bytes,
                                     void *stream) {
    RSC_TRACE("rsc_partitioner_loss_grad");
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!Xb || !T || batch < 1 || !loss_host) return fail(RSC_ERR_INVALID_ARG, "bad arguments");
    size_t need = 0;
    rsc_partitioner_loss_grad_workspace_size(p, batch, &need);
    if (!workspace || workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve cv(workspace);
    cv.take<uint8_t>(kStatusBytes);
    const size_t B = batch;
    TrainBufs b;
    b.Xb = const_cast<float *>(Xb);
    b.T = const_cast<float *>(T);
    b.Z1 = cv.take<float>(B * p->H);
    b.Z2 = cv.take<float>(B * p->H);
    b.dA = cv.take<float>(B * p->H);
    b.dZ = cv.take<float>(B * p->H);
    b.Z3 = cv.take<float>(B * p->P);
    b.dZ3 = cv.take<float>(B * p->P);
    b.grad = grad ? grad : cv.take<float>(p->np);
    b.loss = cv.take<float>(1);
    RSC_CUDA_TRY(cudaMemsetAsync(b.loss, 0, sizeof(float), st));
    mlp_loss_grad(p, st, batch, b);
    RSC_CUDA_TRY(cudaGetLastError());
    float l = 0.f;
    RSC_CUDA_TRY(cudaMemcpyAsync(&l, b.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    rsc_status ks = take_status(p, st);
    if (ks != RSC_OK) return ks;
    *loss_host = l / (float)batch;
    return RSC_OK;
}

}  // extern "C"

// ============================================ training, index and search

namespace {

struct PartLayout {
    unsigned int *status;
    float *Y, *ny, *prep_scratch;   // prep rows of X
    void *Qb, *Db;                  // bf16 operands of X (unsorted)
    // training
    int32_t *labels;                // [n] nearest-centroid part of every row
    float *ksum;                    // [P, d]
    int32_t *kcnt;                  // [P]
    float *Xt;                      // [n_train, d] gathered training rows (FP32)
    int32_t *nbr;                   // [n_train, k] exact neighbours of the training rows
    float *nbr_dist;                // [n_train, k]
    int32_t *order;                 // [n_train] shuffled training positions
    float *Xb, *T, *Z1, *Z2, *Z3, *dZ3, *dA, *dZ, *grad, *loss;
    // segments (parts) of gathered query rows
    int32_t *gcnt, *gcursor;        // [P] each
    int64_t *goff, *doff;           // [P + 1] each
    int32_t *items;                 // [P + 1]
    int32_t *item_counter;          // [1] the probe search's dynamic item counter
    // search (per query chunk)
    int32_t *route;                 // [chunk, R]
    int32_t *gq;                    // [chunk * R]
    int64_t *gpos;                  // [chunk * R]
    void *Qg;                       // [chunk * R, 64] bf16
    int32_t *cand;                  // [chunk * R, kPerSlot]
    float *Xq;                      // [kChunkRows, d] gathered network input
};

PartLayout carve_part(void *ws, const rsc_partitioner *p, int64_t n, int64_t n_train, int k, int64_t chunk, int R,
                      size_t *bytes) {
    Carve cv(ws);
    PartLayout L;
    const int DP = ((p->d + 7) / 8) * 8;
    const int64_t NT = std::max<int64_t>(n_train, 1);
    const int64_t B = 1024;
    const int64_t slots = std::max<int64_t>(chunk * R, NT);
    L.status = cv.take<unsigned int>(kStatusBytes / 4);
    L.Y = cv.take<float>((size_t)n * DP);
    L.ny = cv.take<float>((size_t)n);
    L.prep_scratch = cv.take<float>(prep_scratch_floats());
    L.Qb = cv.take<uint16_t>((size_t)n * 64);
    L.Db = cv.take<uint16_t>((size_t)n * 64);
    L.labels = cv.take<int32_t>((size_t)n);
    L.ksum = cv.take<float>((size_t)p->P * p->d);
    L.kcnt = cv.take<int32_t>((size_t)p->P);
    L.Xt = cv.take<float>((size_t)NT * p->d);
    L.nbr = cv.take<int32_t>((size_t)NT * k);
    L.nbr_dist = cv.take<float>((size_t)NT * k);
    L.order = cv.take<int32_t>((size_t)NT);
    L.Xb = cv.take<float>((size_t)B * p->d);
    L.T = cv.take<float>((size_t)B * p->P);
    L.Z1 = cv.take<float>((size_t)kChunkRows * p->H);
    L.Z2 = cv.take<float>((size_t)kChunkRows * p->H);
    L.Z3 = cv.take<float>((size_t)kChunkRows * p->P);
    L.dZ3 = cv.take<float>((size_t)B * p->P);
    L.dA = cv.take<float>((size_t)B * p->H);
    L.dZ = cv.take<float>((size_t)B * p->H);
    L.grad = cv.take<float>((size_t)p->np);
    L.loss = cv.take<float>(1);
    L.gcnt = cv.take<int32_t>((size_t)p->P * 2);
    L.gcursor = L.gcnt ? L.gcnt + p->P : nullptr;
    L.goff = cv.take<int64_t>((size_t)p->P + 1);
    L.doff = cv.take<int64_t>((size_t)p->P + 1);
    L.items = cv.take<int32_t>((size_t)p->P + 1);
    L.item_counter = cv.take<int32_t>(1);
    L.route = cv.take<int32_t>((size_t)chunk * R);
    L.gq = cv.take<int32_t>((size_t)slots);
    L.gpos = cv.take<int64_t>((size_t)slots);
    L.Qg = cv.take<uint16_t>((size_t)slots * 64);
    L.cand = cv.take<int32_t>((size_t)slots * kPerSlot);
    L.Xq = cv.take<float>((size_t)kChunkRows * p->d);
    if (bytes) *bytes = cv.used;
    return L;
}

int64_t search_chunk(int64_t nq) { return std::min<int64_t>(std::max<int64_t>(nq, 1), 1 << 20); }

// Exact candidates of gathered query rows, segment by segment, through the
// tensor-core kernel (segment p: slots goff[p].. x database rows doff[p]..).
rsc_status probe_search(cudaStream_t st, const void *Dop, int64_t n_db, int64_t n_slots, int P_seg,
                        const PartLayout &L, const int64_t *doff) {
    part::offsets_kernel<<<1, 32, 0, st>>>(P_seg, L.gcnt, L.goff, tck::BM, L.items);
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, L.Qg, std::max<int64_t>(n_slots, 1), 1, tck::BM);
    if (e == cudaSuccess) e = tck::make_map(&md, Dop, n_db, 1, tck::BN);
    if (e != cudaSuccess) return fail(RSC_ERR_CUDA, "tensor map: %s", cudaGetErrorString(e));
    tck::ProbeWork work{P_seg, L.goff, doff, L.items, L.cand, L.item_counter};
    e = cudaMemsetAsync(L.item_counter, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = tck::launch_kernel<1, kSlotList, kSlotParts>(mq, md, work, L.status, st);
    if (e != cudaSuccess) return fail(RSC_ERR_CUDA, "probe search launch: %s", cudaGetErrorString(e));
    return RSC_OK;
}

rsc_status launch_rerank_probe(cudaStream_t st, const float *X, int64_t n_db, int d, const int32_t *qrows,
                               int64_t q_base, int64_t nq, int R, const int64_t *gpos, const int32_t *cand,
                               const int32_t *perm, int k, int32_t *idx, float *dist) {
    int C2 = 32;
    while (C2 < R * kPerSlot) C2 <<= 1;
    if (C2 > 1024) return fail(RSC_ERR_INVALID_ARG, "too many probe candidates");
    const size_t smem = sizeof(float) * part::kRWarps * 64 + (sizeof(float) + sizeof(int)) * part::kRWarps * C2;
    part::rerank_probe_kernel<<<(unsigned)ceil_div(nq, part::kRWarps), part::kRWarps * 32, smem, st>>>(
        X, d, qrows, q_base, nq, R, gpos, cand, kPerSlot, perm, n_db, C2, k, idx, dist);
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

template <int R>
void launch_nearest(cudaStream_t st, const float *X, const int32_t *rows, int64_t npts, int d, const float *C, int P,
                    int32_t *out) {
    part::nearest_centroids_kernel<R><<<(unsigned)ceil_div(npts, 128), 128, 0, st>>>(X, rows, npts, d, C, P, out);
}

void launch_route(cudaStream_t st, int R, const float *X, const int32_t *rows, int64_t npts, int d, const float *C,
                  int P, int32_t *out) {
    switch (R) {
        case 1: launch_nearest<1>(st, X, rows, npts, d, C, P, out); break;
        case 2: launch_nearest<2>(st, X, rows, npts, d, C, P, out); break;
        case 4: launch_nearest<4>(st, X, rows, npts, d, C, P, out); break;
        default: launch_nearest<8>(st, X, rows, npts, d, C, P, out); break;
    }
}

void launch_top_logits(cudaStream_t st, int R, int64_t rows, int P, const float *Z, int32_t *out) {
    const unsigned blocks = (unsigned)ceil_div(rows * 32, 256);
    switch (R) {
        case 1: part::top_logits_kernel<1><<<blocks, 256, 0, st>>>(rows, P, Z, out); break;
        case 2: part::top_logits_kernel<2><<<blocks, 256, 0, st>>>(rows, P, Z, out); break;
        case 4: part::top_logits_kernel<4><<<blocks, 256, 0, st>>>(rows, P, Z, out); break;
        default: part::top_logits_kernel<8><<<blocks, 256, 0, st>>>(rows, P, Z, out); break;
    }
}

// Network top-R parts of `count` rows of X (ids `rows`, or rows 0..count-1).
rsc_status network_route(const rsc_partitioner *p, cudaStream_t st, const float *X, const int32_t *rows,
                         int64_t count, int R, const PartLayout &L, int32_t *out) {
    for (int64_t c0 = 0; c0 < count; c0 += kChunkRows) {
        const int B = (int)std::min<int64_t>(kChunkRows, count - c0);
        const float *xb = X + c0 * p->d;
        if (rows) {
            part::gather_rows_kernel<<<(unsigned)ceil_div((int64_t)B * p->d, 256), 256, 0, st>>>(rows + c0, B, X, p->d,
                                                                                               L.Xq);
            xb = L.Xq;
        }
        mlp_forward(p, st, B, xb, L.Z1, L.Z2, L.Z3, L.status);
        launch_top_logits(st, R, B, p->P, L.Z3, out + c0 * R);
    }
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

int round_probe(int R) { return R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : 8; }

rsc_status prep_operands(const rsc_partitioner *p, cudaStream_t st, const float *X, int64_t n, const PartLayout &L) {
    const int DP = ((p->d + 7) / 8) * 8;
    RSC_CUDA_TRY(launch_prep_fp32(X, n, p->d, DP, RSC_EUCLIDEAN, L.Y, L.ny, L.prep_scratch, st));
    RSC_CUDA_TRY(launch_prep_bf16(L.Y, n, p->d, DP, RSC_EUCLIDEAN, nullptr, L.Qb, L.Db, st));
    return RSC_OK;
}

}  // namespace

extern "C" {

rsc_status rsc_partitioner_workspace_size(const rsc_partitioner *p, int64_t n, int64_t n_train, int32_t k,
                                          int64_t n_queries, int32_t n_probe, size_t *bytes) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!bytes || n < 1 || k < 1 || k > 16 || n_probe < 1 || n_probe > kMaxProbe || n_train < 0 || n_queries < 0)
        return fail(RSC_ERR_INVALID_ARG, "bad sizes (k <= 16, 1 <= n_probe <= 8)");
    carve_part(nullptr, p, n, n_train, k, search_chunk(n_queries), round_probe(n_probe), bytes);
    return RSC_OK;
}

rsc_status rsc_partitioner_build_index(rsc_partitioner *p, const float *X, int64_t n, void *workspace,
                                       size_t workspace_bytes, void *stream) {
    RSC_TRACE("rsc_partitioner_build_index");
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!X || n < 1 || n >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "X / n");
    size_t need = 0;
    rsc_partitioner_workspace_size(p, n, 0, 1, 1, 1, &need);
    if (!workspace || workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PartLayout L = carve_part(workspace, p, n, 0, 1, 1, 1, nullptr);
    if (p->n_db != n) {   // (re)allocate the index arrays owned by the handle
        RSC_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(p->perm);
        cudaFree(p->doff);
        cudaFree(p->Db_sorted);
        p->perm = nullptr;
        p->doff = nullptr;
        p->Db_sorted = nullptr;
        p->n_db = 0;
        RSC_CUDA_TRY(cudaMalloc(&p->perm, sizeof(int32_t) * n));
        RSC_CUDA_TRY(cudaMalloc(&p->doff, sizeof(int64_t) * (p->P + 1)));
        RSC_CUDA_TRY(cudaMalloc(&p->Db_sorted, (size_t)n * 128));
        p->n_db = n;
    }
    if ((s = prep_operands(p, st, X, n, L)) != RSC_OK) return s;
    // every database row goes to the part its network output ranks first
    if ((s = network_route(p, st, X, nullptr, n, 1, L, L.labels)) != RSC_OK) return s;
    RSC_CUDA_TRY(cudaMemsetAsync(L.gcnt, 0, sizeof(int32_t) * p->P * 2, st));
    part::histogram_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, L.labels, L.gcnt);
    part::offsets_kernel<<<1, 32, 0, st>>>(p->P, L.gcnt, p->doff, 1, nullptr);
    part::scatter_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, L.labels, p->doff, L.gcursor, p->perm);
    part::permute_rows_kernel<<<(unsigned)ceil_div(n * 8, 256), 256, 0, st>>>(
        static_cast<const uint4 *>(L.Db), p->perm, n, static_cast<uint4 *>(p->Db_sorted));
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

rsc_status rsc_partitioner_train(rsc_partitioner *p, const float *X, int64_t n, const int32_t *train_rows,
                                 int64_t n_train, int32_t k, int32_t kmeans_iters, int32_t epochs, int32_t batch,
                                 float lr, float *final_loss, void *workspace, size_t workspace_bytes, void *stream) {
    RSC_TRACE("rsc_partitioner_train");
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!X || !train_rows || n < 1 || n >= (int64_t(1) << 31) || n_train < p->P || n_train > n)
        return fail(RSC_ERR_INVALID_ARG, "X / n / train rows (n_parts <= n_train <= n)");
    if (k < 1 || k > 16 || epochs < 0 || batch < 1 || batch > 1024 || batch > n_train || kmeans_iters < 0 ||
        !(lr > 0.f))
        return fail(RSC_ERR_INVALID_ARG, "k <= 16, batch <= min(1024, n_train), lr > 0");
    size_t need = 0;
    rsc_partitioner_workspace_size(p, n, n_train, k, 1, 1, &need);
    if (!workspace || workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PartLayout L = carve_part(workspace, p, n, n_train, k, search_chunk(1), 1, nullptr);
    const int d = p->d, P = p->P;
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));

    // 1. k-means parts on the training rows (initial centroids: the first P of them)
    part::gather_rows_kernel<<<(unsigned)ceil_div((int64_t)P * d, 256), 256, 0, st>>>(train_rows, P, X, d,
                                                                                   p->centroids);
    for (int it = 0; it < kmeans_iters; ++it) {
        launch_route(st, 1, X, train_rows, n_train, d, p->centroids, P, L.labels);
        RSC_CUDA_TRY(cudaMemsetAsync(L.ksum, 0, sizeof(float) * P * d, st));
        RSC_CUDA_TRY(cudaMemsetAsync(L.kcnt, 0, sizeof(int32_t) * P, st));
        part::kmeans_accum_kernel<<<(unsigned)ceil_div(n_train * d, 256), 256, 0, st>>>(X, train_rows, n_train, d,
                                                                                      L.labels, L.ksum, L.kcnt);
        part::kmeans_finalize_kernel<<<(unsigned)ceil_div(P * d, 256), 256, 0, st>>>(P, d, L.ksum, L.kcnt,
                                                                                   p->centroids);
    }
    // the part of every row: its nearest centroid (the targets' labels)
    launch_route(st, 1, X, nullptr, n, d, p->centroids, P, L.labels);

    // 2. exact k nearest neighbours of the training rows among all n rows:
    //    one segment = every training row (gathered) x the whole database
    if ((s = prep_operands(p, st, X, n, L)) != RSC_OK) return s;
    part::permute_rows_kernel<<<(unsigned)ceil_div(n_train * 8, 256), 256, 0, st>>>(
        static_cast<const uint4 *>(L.Qb), train_rows, n_train, static_cast<uint4 *>(L.Qg));
    part::set_segment_kernel<<<1, 1, 0, st>>>(L.gcnt, (int32_t)n_train, L.doff, 0, n);
    if ((s = probe_search(st, L.Db, n, n_train, 1, L, L.doff)) != RSC_OK) return s;
    part::iota64_kernel<<<(unsigned)ceil_div(n_train, 256), 256, 0, st>>>(n_train, L.gpos);
    if ((s = launch_rerank_probe(st, X, n, d, train_rows, 0, n_train, 1, L.gpos, L.cand, nullptr, k, L.nbr,
                                 L.nbr_dist)) != RSC_OK)
        return s;
    part::gather_rows_kernel<<<(unsigned)ceil_div(n_train * d, 256), 256, 0, st>>>(train_rows, n_train, X, d, L.Xt);

    // 3. minibatch training on soft targets (histogram of the neighbours' parts), Adam
    std::vector<int32_t> order(n_train);
    std::mt19937_64 gen(p->seed ^ 0x9e3779b97f4a7c15ull);
    TrainBufs b{L.Xb, L.T, L.Z1, L.Z2, L.Z3, L.dZ3, L.dA, L.dZ, L.grad, L.loss};
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float epoch_loss = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n_train; ++i) order[i] = (int32_t)i;
        std::shuffle(order.begin(), order.end(), gen);
        RSC_CUDA_TRY(cudaMemcpyAsync(L.order, order.data(), sizeof(int32_t) * n_train, cudaMemcpyHostToDevice, st));
        RSC_CUDA_TRY(cudaMemsetAsync(L.loss, 0, sizeof(float), st));
        int64_t rows_seen = 0;
        for (int64_t b0 = 0; b0 + batch <= n_train; b0 += batch) {
            const int B = batch;
            const int32_t *pos = L.order + b0;
            part::gather_rows_kernel<<<(unsigned)ceil_div((int64_t)B * d, 256), 256, 0, st>>>(pos, B, L.Xt, d, L.Xb);
            RSC_CUDA_TRY(cudaMemsetAsync(L.T, 0, sizeof(float) * (size_t)B * P, st));
            part::targets_kernel<<<(unsigned)ceil_div((int64_t)B * k, 256), 256, 0, st>>>(B, k, pos, L.nbr, L.labels,
                                                                                       P, L.T);
            mlp_loss_grad(p, st, B, b);
            ++p->step;
            const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
            part::adam_kernel<<<(unsigned)ceil_div(p->np, 256), 256, 0, st>>>(p->np, p->params, L.grad, p->adam_m,
                                                                           p->adam_v, lr, b1, b2, eps, c1, c2);
            rows_seen += B;
        }
        RSC_CUDA_TRY(cudaGetLastError());
        float l = 0.f;
        RSC_CUDA_TRY(cudaMemcpyAsync(&l, L.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        RSC_CUDA_TRY(cudaStreamSynchronize(st));   // `order` is rewritten next epoch
        epoch_loss = rows_seen ? l / (float)rows_seen : 0.f;
    }
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    rsc_status ks = take_status(p, st);
    if (ks != RSC_OK) return ks;
    if (final_loss) *final_loss = epoch_loss;
    // 4. index the database by the trained network
    return rsc_partitioner_build_index(p, X, n, workspace, workspace_bytes, stream);
}

rsc_status rsc_knn_partitioned(rsc_partitioner *p, const float *X, int64_t n, int32_t k, int32_t n_probe,
                               int32_t routing, const int32_t *query_rows, int64_t n_queries, int32_t *idx,
                               float *dist, void *workspace, size_t workspace_bytes, void *stream) {
    RSC_TRACE("rsc_knn_partitioned");
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!X || !idx || !dist || n != p->n_db) return fail(RSC_ERR_INVALID_ARG, "X / outputs / n (index built for n=%lld)",
                                                        (long long)p->n_db);
    if (k < 1 || k > kSlotList || (n_probe != 1 && n_probe != 2 && n_probe != 4 && n_probe != 8) ||
        (routing != 0 && routing != 1))
        return fail(RSC_ERR_INVALID_ARG, "k <= 16, n_probe in {1, 2, 4, 8}, routing 0 (network) or 1 (centroids)");
    const int64_t nq = query_rows ? n_queries : n;
    if (nq < 0) return fail(RSC_ERR_INVALID_ARG, "n_queries");
    size_t need = 0;
    rsc_partitioner_workspace_size(p, n, 0, k, nq, n_probe, &need);
    if (!workspace || workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int R = n_probe;
    const int64_t chunk = search_chunk(nq);
    PartLayout L = carve_part(workspace, p, n, 0, k, chunk, round_probe(R), nullptr);
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));
    if ((s = prep_operands(p, st, X, n, L)) != RSC_OK) return s;
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t cq = std::min<int64_t>(chunk, nq - q0);
        const int32_t *rows = query_rows ? query_rows + q0 : nullptr;   // else rows q0 .. q0 + cq - 1
        // 1. route each query to R parts
        if (routing == 0) {
            if (rows) s = network_route(p, st, X, rows, cq, R, L, L.route);
            else s = network_route(p, st, X + q0 * p->d, nullptr, cq, R, L, L.route);
            if (s != RSC_OK) return s;
        } else {
            if (rows) launch_route(st, R, X, rows, cq, p->d, p->centroids, p->P, L.route);
            else launch_route(st, R, X + q0 * p->d, nullptr, cq, p->d, p->centroids, p->P, L.route);
        }
        // 2. group (query, probe) pairs by part; gather the query operand rows
        RSC_CUDA_TRY(cudaMemsetAsync(L.gcnt, 0, sizeof(int32_t) * p->P * 2, st));
        part::histogram_kernel<<<(unsigned)ceil_div(cq * R, 256), 256, 0, st>>>(cq * R, L.route, L.gcnt);
        part::offsets_kernel<<<1, 32, 0, st>>>(p->P, L.gcnt, L.goff, tck::BM, L.items);
        part::probe_scatter_kernel<<<(unsigned)ceil_div(cq * R, 256), 256, 0, st>>>(cq, R, L.route, L.goff,
                                                                                   L.gcursor, L.gq, L.gpos);
        // gq holds chunk-local query positions: make them rows of X
        const int64_t slots = cq * R;
        if (rows) part::compose_kernel<<<(unsigned)ceil_div(slots, 256), 256, 0, st>>>(slots, L.gq, rows, L.gq);
        else part::add_offset_kernel<<<(unsigned)ceil_div(slots, 256), 256, 0, st>>>(slots, L.gq, (int32_t)q0);
        part::permute_rows_kernel<<<(unsigned)ceil_div(slots * 8, 256), 256, 0, st>>>(
            static_cast<const uint4 *>(L.Qb), L.gq, slots, static_cast<uint4 *>(L.Qg));
        // 3. each part's gathered queries against that part's database rows
        if ((s = probe_search(st, p->Db_sorted, n, slots, p->P, L, p->doff)) != RSC_OK) return s;
        // 4. merge the probed parts' candidates with the exact FP32 re-rank
        if ((s = launch_rerank_probe(st, X, n, p->d, rows, q0, cq, R, L.gpos, L.cand, p->perm, k, idx + q0 * k,
                                     dist + q0 * k)) != RSC_OK)
            return s;
    }
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

rsc_status rsc_partitioner_save(const rsc_partitioner *p, const char *path) {
    rsc_status s = check_handle(p);
    if (s != RSC_OK) return s;
    if (!path) return fail(RSC_ERR_INVALID_ARG, "path is NULL");
    std::vector<float> params(p->np), cent((size_t)p->P * p->d);
    RSC_CUDA_TRY(cudaMemcpy(params.data(), p->params, sizeof(float) * p->np, cudaMemcpyDeviceToHost));
    RSC_CUDA_TRY(cudaMemcpy(cent.data(), p->centroids, sizeof(float) * cent.size(), cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(RSC_ERR_INVALID_ARG, "cannot open %s", path);
    const int32_t hdr[6] = {0x52534350, 1, p->d, p->P, p->H, p->bf16};   // "RSCP", version 1
    bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&p->seed, sizeof(p->seed), 1, f) == 1 &&
              fwrite(params.data(), sizeof(float), params.size(), f) == params.size() &&
              fwrite(cent.data(), sizeof(float), cent.size(), f) == cent.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? RSC_OK : fail(RSC_ERR_INVALID_ARG, "write to %s failed", path);
}

rsc_status rsc_partitioner_load(const char *path, rsc_partitioner **out) {
    if (!path || !out) return fail(RSC_ERR_INVALID_ARG, "path / out is NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(RSC_ERR_INVALID_ARG, "cannot open %s", path);
    int32_t hdr[6];
    uint64_t seed = 0;
    if (fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 0x52534350 || hdr[1] != 1 ||
        fread(&seed, sizeof(seed), 1, f) != 1) {
        fclose(f);
        return fail(RSC_ERR_INVALID_ARG, "%s is not a partitioner file", path);
    }
    rsc_partitioner *p = nullptr;
    rsc_status s = rsc_partitioner_create(hdr[2], hdr[3], hdr[4], hdr[5], seed, &p);
    if (s != RSC_OK) {
        fclose(f);
        return s;
    }
    std::vector<float> params(p->np), cent((size_t)p->P * p->d);
    const bool ok = fread(params.data(), sizeof(float), params.size(), f) == params.size() &&
                    fread(cent.data(), sizeof(float), cent.size(), f) == cent.size();
    fclose(f);
    if (!ok) {
        rsc_partitioner_destroy(p);
        return fail(RSC_ERR_INVALID_ARG, "%s is truncated", path);
    }
    cudaError_t e = cudaMemcpy(p->params, params.data(), sizeof(float) * p->np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->centroids, cent.data(), sizeof(float) * cent.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rsc_partitioner_destroy(p);
        return fail(RSC_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return RSC_OK;
}

}  // extern "C"
