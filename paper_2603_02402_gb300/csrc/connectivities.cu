// Fuzzy connectivities of a kNN graph, in FP32 on the GPU.
//
// The paper stores the neighbourhood graph in .obsp for UMAP and Leiden
// (Methods, "Dimensionality reduction and graph analysis") and follows scanpy
// (Methods, "Implementation"), whose graph is the UMAP fuzzy simplicial set:
//   rho_i   = first non-zero kNN distance of row i,
//   sigma_i : sum_{c=1}^{k-1} exp(-max(0, d_ic - rho_i)/sigma_i) = log2 k
//             (64 bisection steps, stop within 1e-5, floor 1e-3 * mean),
//   w_ic    = 0 (self), 1 (d <= rho or sigma == 0), else exp(-(d - rho)/sigma),
//   G       = A + A^T - A o A^T, no diagonal, no zeros, CSR, sorted columns.
//
// Phases (k <= 32: a group of 16 or 32 lanes per row, one lane per kNN
// entry, so every row-wise loop is a lane-parallel step; k > 32: a warp or a
// thread per row):
//   mean      deterministic two-level sum of all distances (for rho == 0 rows)
//   smooth    rho, sigma, weights (thread per row: the bisection is
//             arithmetic); the row's (column, weight) pairs sorted by column
//             into 16-byte rows of KP slots
//   count     per edge i->j: is i in row j's list (the partner row read whole
//             with vector loads); own entry value a + b - ab; edges whose
//             reverse is absent also go to row j (in-degree atomics)
//   scan      row pointers (int64)
//   fill      own entries in column order (ballot prefix), transposed entries
//             via per-row atomic cursors (the scatter-add-with-atomics idea of
//             the paper's categorical aggregation kernels, Methods, "Custom
//             GPU kernels")
//   sort      rows that received transposed entries are sorted by column
//             (a thread in registers up to 32 entries, a warp in shared
//             memory up to 512, a block per row beyond)
#include <limits.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kStatusCapacity = RSC_ERR_CAPACITY;

// ------------------------------------------------------------------ mean

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ float block_sum(float v, float *red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads)
mean_partials_kernel(const float *__restrict__ dist, int64_t total, float *__restrict__ partials) {
    __shared__ float red[kThreads];
    const int64_t chunk = ceil_div(total, gridDim.x);
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(total, begin + chunk);
    float s = 0.f, c = 0.f;
    for (int64_t e = begin + threadIdx.x; e < end; e += blockDim.x) kahan_add(s, c, dist[e]);
    const float r = block_sum(s - c, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kMeanBlocks)
mean_final_kernel(const float *__restrict__ partials, int64_t total, float *__restrict__ mean_all) {
    __shared__ float red[kMeanBlocks];
    const float r = block_sum(partials[threadIdx.x], red);
    if (threadIdx.x == 0) mean_all[0] = (float)((double)r / (double)total);
}

// ---------------------------------------------------------------- smooth

constexpr float kTol = 1e-5f;
constexpr int kIters = 64;
constexpr float kFloor = 1e-3f;

// One warp per row, 32 < k <= 256 (up to 8 entries per lane).
constexpr int kWarpRows = 4;
constexpr int kWarpMaxK = 256;

__global__ void __launch_bounds__(kWarpRows * 32)
smooth_warp_kernel(const int32_t *__restrict__ idx, const float *__restrict__ dist, int64_t n,
                   int k, const float *__restrict__ mean_all, float *__restrict__ rho_out,
                   float *__restrict__ sigma_out, int32_t *__restrict__ scol,
                   float *__restrict__ sw) {
    __shared__ int s_col[kWarpRows][kWarpMaxK];
    __shared__ float s_w[kWarpRows][kWarpMaxK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarpRows + warp;
    if (i >= n) return;
    constexpr int E = kWarpMaxK / 32;
    float dd[E];
    int col[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        dd[e] = (c < k) ? dist[i * k + c] : 0.f;
        col[e] = (c < k) ? idx[i * k + c] : INT_MAX;
    }
    // rho: the non-zero distance with the smallest column position
    int first = INT_MAX;
#pragma unroll
    for (int e = E - 1; e >= 0; --e) {
        const int c = lane + 32 * e;
        if (c < k && dd[e] > 0.f) first = c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, off));
    float mine = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (lane + 32 * e == first) mine = dd[e];
    const float r = (first != INT_MAX) ? __shfl_sync(0xffffffffu, mine, first % 32) : 0.f;

    const float target = log2f((float)k);
    float lo = 0.f, hi = INFINITY, mid = 1.f;
    for (int it = 0; it < kIters; ++it) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = lane + 32 * e;
            if (c >= 1 && c < k) {
                const float g = dd[e] - r;
                s += (g > 0.f) ? expf(-(g / mid)) : 1.f;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const float psum = s;   // identical on every lane (commutative butterfly)
        if (fabsf(psum - target) < kTol) break;
        const float prev = mid;
        if (psum > target) {
            hi = mid;
            mid = (lo + hi) * 0.5f;
        } else {
            lo = mid;
            mid = isinf(hi) ? mid * 2.f : (lo + hi) * 0.5f;
        }
        // a repeated midpoint is a fixed point (same sum, same branch, same
        // bounds): the remaining steps would not move it
        if (mid == prev) break;
    }
    float rs = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) rs += (lane + 32 * e < k) ? dd[e] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, off);
    const float floor_v = (r > 0.f) ? kFloor * (rs / (float)k) : kFloor * mean_all[0];
    const float sig = (mid < floor_v) ? floor_v : mid;
    if (lane == 0) {
        rho_out[i] = r;
        sigma_out[i] = sig;
    }
    int P = 32;
    while (P < k) P <<= 1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        if (c >= P) continue;
        float v;
        if ((int64_t)col[e] == i) v = 0.f;
        else if (dd[e] - r <= 0.f || sig == 0.f) v = 1.f;
        else v = expf(-((dd[e] - r) / sig));
        int cc = col[e];
        if (cc < 0 || (int64_t)cc >= n || c >= k) {   // empty or malformed slot
            cc = INT_MAX;
            v = 0.f;
        }
        s_col[warp][c] = cc;
        s_w[warp][c] = v;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < P / 2; t += 32) {
                const int a = (t / stride) * 2 * stride + (t % stride), b = a + stride;
                const bool asc = (a & size) == 0;
                const int ca = s_col[warp][a], cb = s_col[warp][b];
                if ((ca > cb) == asc) {
                    s_col[warp][a] = cb;
                    s_col[warp][b] = ca;
                    const float tw = s_w[warp][a];
                    s_w[warp][a] = s_w[warp][b];
                    s_w[warp][b] = tw;
                }
            }
            __syncwarp();
        }
    }
    for (int c = lane; c < k; c += 32) {
        scol[i * k + c] = s_col[warp][c];
        sw[i * k + c] = s_w[warp][c];
    }
}

// ----------------------------------------------------------------- count

__device__ __forceinline__ float fuzzy_union(float a, float b) {
    // a + b - a*b, rounded the same way whichever endpoint computes it
    return __fsub_rn(__fadd_rn(a, b), __fmul_rn(a, b));
}

__global__ void __launch_bounds__(kThreads)
count_kernel(int64_t n, int k, const int32_t *__restrict__ scol, const float *__restrict__ sw,
             float *__restrict__ gv, int32_t *__restrict__ own_cnt, int32_t *__restrict__ in_cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int own = 0;
    for (int c = 0; c < k; ++c) {
        const int32_t j = scol[i * k + c];
        float out = 0.f;
        if (j != INT_MAX && (int64_t)j != i) {
            const float a = sw[i * k + c];
            const int32_t *rj = scol + (int64_t)j * k;
            int lo = 0, hi = k;
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if ((int64_t)rj[m] < i) lo = m + 1;
                else hi = m;
            }
            const bool mutual = lo < k && (int64_t)rj[lo] == i;
            const float b = mutual ? sw[(int64_t)j * k + lo] : 0.f;
            const float g = fuzzy_union(a, b);
            if (!mutual && a != 0.f) {
                atomicAdd(in_cnt + j, 1);
                out = -g;   // negative marks "also emit the transposed entry"
            } else {
                out = g;
            }
            own += (g != 0.f);
        }
        gv[i * k + c] = out;
    }
    own_cnt[i] = own;
}

// ------------------------------------------ lane-per-entry kernels (k <= 32)
//
// A row is handled by a group of G lanes (G = 16 for k <= 16, 32 for
// k <= 32), lane c holding entry c; 32 / G rows per warp.  Row reductions
// are xor butterflies inside the group (every lane gets the same sum) and
// the row's (column, weight) pairs are sorted by a shuffle bitonic network.

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Ascending bitonic sort of one (col, w) pair per lane across each G-lane
// group (lane c of the group ends with the c-th smallest column).
template <int G>
__device__ __forceinline__ void group_sort_by_col(int &col, float &w, int c) {
#pragma unroll
    for (int size = 2; size <= G; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int pc = __shfl_xor_sync(0xffffffffu, col, stride);
            const float pw = __shfl_xor_sync(0xffffffffu, w, stride);
            const bool asc = (c & size) == 0;
            const bool lower = (c & stride) == 0;
            const bool take = (lower == asc) ? (pc < col) : (pc > col);
            if (take) {
                col = pc;
                w = pw;
            }
        }
    }
}

// Bitonic sort of KM (column, weight) pairs held in registers, by column.
template <int KM>
__device__ __forceinline__ void sort_pairs_by_col(int (&col)[KM], float (&w)[KM]) {
#pragma unroll
    for (int size = 2; size <= KM; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int i = 0; i < KM; ++i) {
                const int p = i ^ stride;
                if (p > i) {
                    const bool asc = (i & size) == 0;
                    if ((col[i] > col[p]) == asc) {
                        const int tc = col[i];
                        col[i] = col[p];
                        col[p] = tc;
                        const float tw = w[i];
                        w[i] = w[p];
                        w[p] = tw;
                    }
                }
            }
        }
    }
}

// Thread per row, k <= KM (16 or 32): the bisection is arithmetic-bound, so
// each thread runs its own row's loop (no cross-lane reductions per step).
// exp(-g / sigma) is evaluated as exp2(g * (-log2(e) / sigma)) with one
// reciprocal per step.  Output rows of KP slots are 16-byte aligned and
// written with vector stores.
template <int KM>
__global__ void __launch_bounds__(kThreads)
smooth_row_kernel(const int32_t *__restrict__ idx, const float *__restrict__ dist, int64_t n, int k, int KP,
                  const float *__restrict__ mean_all, float *__restrict__ rho_out, float *__restrict__ sigma_out,
                  int32_t *__restrict__ scol, float *__restrict__ sw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float dd[KM];
    int col[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) {
        dd[c] = (c < k) ? dist[i * k + c] : 0.f;
        col[c] = (c < k) ? idx[i * k + c] : INT_MAX;
    }
    float r = 0.f;
    bool found = false;
#pragma unroll
    for (int c = 0; c < KM; ++c) {
        if (c < k && !found && dd[c] > 0.f) {
            r = dd[c];
            found = true;
        }
    }
    float g[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) g[c] = dd[c] - r;
    const float target = log2f((float)k);
    constexpr float kNegLog2e = -1.4426950408889634f;
    float lo = 0.f, hi = INFINITY, mid = 1.f;
    for (int it = 0; it < kIters; ++it) {
        const float sc = kNegLog2e / mid;
        float s = 0.f, comp = 0.f;   // Neumaier-compensated sum
#pragma unroll
        for (int c = 1; c < KM; ++c) {
            if (c < k) {
                const float t = (g[c] > 0.f) ? exp2f(g[c] * sc) : 1.f;
                const float u = s + t;
                comp += (fabsf(s) >= fabsf(t)) ? ((s - u) + t) : ((t - u) + s);
                s = u;
            }
        }
        const float psum = s + comp;
        if (fabsf(psum - target) < kTol) break;
        const float prev = mid;
        if (psum > target) {
            hi = mid;
            mid = (lo + hi) * 0.5f;
        } else {
            lo = mid;
            mid = isinf(hi) ? mid * 2.f : (lo + hi) * 0.5f;
        }
        // a repeated midpoint is a fixed point (same sum, same branch, same
        // bounds): the remaining steps would not move it
        if (mid == prev) break;
    }
    float row_sum = 0.f;
#pragma unroll
    for (int c = 0; c < KM; ++c) row_sum += (c < k) ? dd[c] : 0.f;
    const float floor_v = (r > 0.f) ? kFloor * (row_sum / (float)k) : kFloor * mean_all[0];
    const float sig = (mid < floor_v) ? floor_v : mid;
    rho_out[i] = r;
    sigma_out[i] = sig;

    float w[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) {
        float v;
        if ((int64_t)col[c] == i) v = 0.f;
        else if (g[c] <= 0.f || sig == 0.f) v = 1.f;
        else v = expf(-(g[c] / sig));
        if (col[c] < 0 || (int64_t)col[c] >= n || c >= k) {   // empty or malformed slot
            col[c] = INT_MAX;
            v = 0.f;
        }
        w[c] = v;
    }
    sort_pairs_by_col<KM>(col, w);
    int4 *oc = reinterpret_cast<int4 *>(scol + i * KP);
    float4 *ow = reinterpret_cast<float4 *>(sw + i * KP);
#pragma unroll
    for (int u = 0; u < KM / 4; ++u) {
        if (4 * u < KP) {
            oc[u] = make_int4(col[4 * u], col[4 * u + 1], col[4 * u + 2], col[4 * u + 3]);
            ow[u] = make_float4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
        }
    }
}

// Lane per own entry i -> j: is i in row j's list?  The partner row (KP
// columns, 16-byte aligned) is read with int4 loads and compared whole.
template <int G>
__global__ void __launch_bounds__(kThreads)
count_group_kernel(int64_t n, int KP, const int32_t *__restrict__ scol, const float *__restrict__ sw,
                   float *__restrict__ gv, int32_t *__restrict__ tslot, int32_t *__restrict__ own_cnt,
                   int32_t *__restrict__ in_cnt) {
    const int lane = threadIdx.x & 31, c = lane & (G - 1), base = lane & ~(G - 1);
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / G) + lane / G;
    const bool row_ok = i < n;
    const bool has = row_ok && c < KP;
    const int32_t j = has ? scol[i * KP + c] : INT_MAX;
    float out = 0.f;
    if (j != INT_MAX && (int64_t)j != i) {
        const float a = sw[i * KP + c];
        const int4 *rj = reinterpret_cast<const int4 *>(scol + (int64_t)j * KP);
        int pos = -1;
#pragma unroll
        for (int u = 0; u < G / 4; ++u) {
            if (4 * u < KP) {
                const int4 q = __ldg(rj + u);
                if ((int64_t)q.x == i) pos = 4 * u;
                if ((int64_t)q.y == i) pos = 4 * u + 1;
                if ((int64_t)q.z == i) pos = 4 * u + 2;
                if ((int64_t)q.w == i) pos = 4 * u + 3;
            }
        }
        const bool mutual = pos >= 0;
        const float b = mutual ? sw[(int64_t)j * KP + pos] : 0.f;
        const float g = fuzzy_union(a, b);
        if (!mutual && a != 0.f) {
            tslot[i * KP + c] = atomicAdd(in_cnt + j, 1);   // its place among row j's transposed entries
            out = -g;   // negative marks "also emit the transposed entry"
        } else {
            out = g;
        }
    }
    if (has) gv[i * KP + c] = out;
    const unsigned own = (__ballot_sync(0xffffffffu, out != 0.f) >> base) & (G == 32 ? 0xffffffffu : ((1u << G) - 1));
    if (row_ok && c == 0) own_cnt[i] = __popc(own);
}

// Lane per own entry: own entries at indptr[i] + (rank among the row's
// non-zero entries), in column order; a transposed entry at its slot (taken
// by the count pass) after the receiving row's own entries.
template <int G>
__global__ void __launch_bounds__(kThreads)
fill_group_kernel(int64_t n, int KP, const int64_t *__restrict__ indptr, const int32_t *__restrict__ scol,
                  const float *__restrict__ gv, const int32_t *__restrict__ own_cnt, const int32_t *__restrict__ tslot,
                  int32_t *__restrict__ indices, float *__restrict__ data, int64_t cap, unsigned int *status) {
    const int lane = threadIdx.x & 31, c = lane & (G - 1), base = lane & ~(G - 1);
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / G) + lane / G;
    const bool has = i < n && c < KP;
    const float v = has ? gv[i * KP + c] : 0.f;
    const unsigned nzm = (__ballot_sync(0xffffffffu, v != 0.f) >> base);
    if (v == 0.f) return;
    const int32_t j = scol[i * KP + c];
    const int64_t p = indptr[i] + __popc(nzm & ((1u << c) - 1));
    if (p < cap) {
        indices[p] = j;
        data[p] = fabsf(v);
    } else {
        record_status(status, kStatusCapacity);
    }
    if (v < 0.f) {
        const int64_t q = indptr[j] + own_cnt[j] + tslot[i * KP + c];
        if (q < cap) {
            indices[q] = (int32_t)i;
            data[q] = -v;
        } else {
            record_status(status, kStatusCapacity);
        }
    }
}

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x / 32;
        int64_t s = (lane < nw) ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int64_t warp_off = (warp > 0) ? warp_sums[warp - 1] : 0;
    total = warp_sums[blockDim.x / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_local_kernel(int64_t n, const int32_t *__restrict__ own_cnt, const int32_t *__restrict__ in_cnt,
                  int64_t *__restrict__ indptr, int64_t *__restrict__ part) {
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const int64_t i = base + e;
        v[e] = (i < n) ? (int64_t)own_cnt[i] + (int64_t)in_cnt[i] : 0;
        sum += v[e];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(sum, warp_sums, total);
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const int64_t i = base + e;
        if (i < n) indptr[i] = run;
        run += v[e];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024)
scan_part_kernel(int64_t nb, int64_t *__restrict__ part, int64_t n, int64_t *__restrict__ indptr) {
    __shared__ int64_t warp_sums[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = (b < nb) ? part[b] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, warp_sums, total);
        if (b < nb) part[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) indptr[n] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_add_kernel(int64_t n, const int64_t *__restrict__ part, int64_t *__restrict__ indptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) indptr[i] += part[i / kScanTile];
}

// ------------------------------------------------------------------ fill

__global__ void __launch_bounds__(kThreads)
fill_kernel(int64_t n, int k, const int64_t *__restrict__ indptr, const int32_t *__restrict__ scol,
            const float *__restrict__ gv, const int32_t *__restrict__ own_cnt,
            int32_t *__restrict__ cursor, int32_t *__restrict__ indices, float *__restrict__ data,
            int64_t cap, unsigned int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = indptr[i];
    for (int c = 0; c < k; ++c) {
        const float v = gv[i * k + c];
        if (v == 0.f) continue;
        const int32_t j = scol[i * k + c];
        if (p < cap) {
            indices[p] = j;
            data[p] = fabsf(v);
        } else {
            record_status(status, kStatusCapacity);
        }
        ++p;
        if (v < 0.f) {
            const int slot = atomicAdd(cursor + j, 1);
            const int64_t q = indptr[j] + own_cnt[j] + slot;
            if (q < cap) {
                indices[q] = (int32_t)i;
                data[q] = -v;
            } else {
                record_status(status, kStatusCapacity);
            }
        }
    }
}

// ------------------------------------------------------------------ sort

constexpr int kSortWarps = 8;
constexpr int kWarpSortMax = 512;
constexpr int kBlockSortMax = 4096;

// Ascending-only bitonic network ("mirrored" first step of each merge), on a
// virtual power-of-two length P = 2^lp >= L; slots at or past L act as +inf
// and the comparators never move them, so no padding needs to be stored.
// Index arithmetic is 32-bit shifts and masks (rows hold < 2^31 entries).
template <class Get, class Put, class Sync>
__device__ void mirrored_bitonic(int L, int lp, int t0, int dt, Get get, Put put, Sync sync) {
    auto cas = [&](int lo, int hi) {
        if (hi >= L) return;
        int ca, cb;
        float wa, wb;
        get(lo, ca, wa);
        get(hi, cb, wb);
        if (ca > cb) {
            put(lo, cb, wb);
            put(hi, ca, wa);
        }
    };
    const int halfP = (1 << lp) >> 1;
    for (int ls = 1; ls <= lp; ++ls) {          // size = 2^ls
        const int lh = ls - 1, half = 1 << lh;
        for (int t = t0; t < halfP; t += dt) {
            const int blk = t >> lh, off = t & (half - 1);
            cas((blk << ls) + off, (blk << ls) + (1 << ls) - 1 - off);
        }
        sync();
        for (int lst = ls - 2; lst >= 0; --lst) {   // stride = 2^lst
            const int stride = 1 << lst;
            for (int t = t0; t < halfP; t += dt) {
                const int lo = ((t >> lst) << (lst + 1)) + (t & (stride - 1));
                cas(lo, lo + stride);
            }
            sync();
        }
    }
}

__device__ __forceinline__ int ceil_log2(int L) {
    int lp = 0;
    while ((1 << lp) < L) ++lp;
    return lp;
}

// Rows that received transposed entries are re-sorted by column.  Thread
// per row for the common short rows (up to 32 entries: loaded and sorted in
// registers, so a warp keeps 32 rows' loads in flight); longer rows are
// queued: up to kWarpSortMax entries for a warp in shared memory, beyond
// that for a block.
__global__ void __launch_bounds__(kThreads)
sort_short_rows_kernel(int64_t n, const int64_t *__restrict__ indptr, const int32_t *__restrict__ in_cnt,
                       int32_t *__restrict__ indices, float *__restrict__ data, int64_t cap,
                       int32_t *__restrict__ mid_rows, int32_t *__restrict__ mid_count,
                       int32_t *__restrict__ long_rows, int32_t *__restrict__ long_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || in_cnt[i] == 0) return;
    const int64_t b = indptr[i], e = indptr[i + 1];
    if (e > cap) return;   // capacity error already recorded by the fill
    const int L = (int)(e - b);
    if (L > 32) {
        if (L <= kWarpSortMax) mid_rows[atomicAdd(mid_count, 1)] = (int32_t)i;
        else long_rows[atomicAdd(long_count, 1)] = (int32_t)i;
        return;
    }
    int col[32];
    float w[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        col[t] = (t < L) ? indices[b + t] : INT_MAX;
        w[t] = (t < L) ? data[b + t] : 0.f;
    }
    if (L <= 16) {
        int c16[16];
        float w16[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            c16[t] = col[t];
            w16[t] = w[t];
        }
        sort_pairs_by_col<16>(c16, w16);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            col[t] = c16[t];
            w[t] = w16[t];
        }
    } else {
        sort_pairs_by_col<32>(col, w);
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        if (t < L) {
            indices[b + t] = col[t];
            data[b + t] = w[t];
        }
    }
}

// Warp per queued row of 33 .. kWarpSortMax entries, in shared memory.
__global__ void __launch_bounds__(kSortWarps * 32)
sort_mid_rows_kernel(const int64_t *__restrict__ indptr, int32_t *__restrict__ indices, float *__restrict__ data,
                     const int32_t *__restrict__ mid_rows, const int32_t *__restrict__ mid_count) {
    __shared__ int s_col[kSortWarps][kWarpSortMax];
    __shared__ float s_w[kSortWarps][kWarpSortMax];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = *mid_count;
    int *sc = s_col[warp];
    float *sv = s_w[warp];
    for (int r = blockIdx.x * kSortWarps + warp; r < cnt; r += gridDim.x * kSortWarps) {
        const int64_t i = mid_rows[r];
        const int64_t b = indptr[i];
        const int L = (int)(indptr[i + 1] - b);
        for (int t = lane; t < L; t += 32) {
            sc[t] = indices[b + t];
            sv[t] = data[b + t];
        }
        __syncwarp();
        mirrored_bitonic(
            L, ceil_log2(L), lane, 32,
            [&](int x, int &c, float &w) { c = sc[x]; w = sv[x]; },
            [&](int x, int c, float w) { sc[x] = c; sv[x] = w; },
            [] { __syncwarp(); });
        for (int t = lane; t < L; t += 32) {
            indices[b + t] = sc[t];
            data[b + t] = sv[t];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024)
sort_long_rows_kernel(const int64_t *__restrict__ indptr, int32_t *__restrict__ indices,
                      float *__restrict__ data, const int32_t *__restrict__ long_rows,
                      const int32_t *__restrict__ long_count) {
    __shared__ int s_col[kBlockSortMax];
    __shared__ float s_w[kBlockSortMax];
    const int cnt = *long_count;
    for (int r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = long_rows[r];
        const int64_t b = indptr[i];
        const int L = (int)(indptr[i + 1] - b);
        const int lp = ceil_log2(L);
        if (L <= kBlockSortMax) {
            for (int t = threadIdx.x; t < L; t += blockDim.x) {
                s_col[t] = indices[b + t];
                s_w[t] = data[b + t];
            }
            __syncthreads();
            mirrored_bitonic(
                L, lp, threadIdx.x, blockDim.x,
                [&](int x, int &c, float &w) { c = s_col[x]; w = s_w[x]; },
                [&](int x, int c, float w) { s_col[x] = c; s_w[x] = w; },
                [] { __syncthreads(); });
            for (int t = threadIdx.x; t < L; t += blockDim.x) {
                indices[b + t] = s_col[t];
                data[b + t] = s_w[t];
            }
        } else {
            int32_t *gc = indices + b;
            float *gw = data + b;
            mirrored_bitonic(
                L, lp, threadIdx.x, blockDim.x,
                [&](int x, int &c, float &w) { c = gc[x]; w = gw[x]; },
                [&](int x, int c, float w) { gc[x] = c; gw[x] = w; },
                [] { __threadfence_block(); __syncthreads(); });
        }
        __syncthreads();
    }
}

}  // namespace

size_t conn_scan_blocks(int64_t n) { return (size_t)ceil_div(n, kScanTile); }

cudaError_t launch_conn_count(const int32_t *idx, const float *dist, int64_t n, int k,
                              int64_t *indptr, const ConnWork &w, cudaStream_t st) {
    const int64_t total = n * (int64_t)k;
    mean_partials_kernel<<<kMeanBlocks, kThreads, 0, st>>>(dist, total, w.partials);
    mean_final_kernel<<<1, kMeanBlocks, 0, st>>>(w.partials, total, w.mean_all);
    const unsigned row_blocks = (unsigned)ceil_div(n, kThreads);
    const int KP = conn_stride(k);
    const unsigned g16_blocks = (unsigned)ceil_div(n, kThreads / 16), g32_blocks = (unsigned)ceil_div(n, kThreads / 32);
    if (k <= 16) {
        smooth_row_kernel<16><<<row_blocks, kThreads, 0, st>>>(idx, dist, n, k, KP, w.mean_all, w.rho, w.sigma,
                                                               w.scol, w.sw);
        count_group_kernel<16><<<g16_blocks, kThreads, 0, st>>>(n, KP, w.scol, w.sw, w.gv, w.tslot, w.own_cnt,
                                                                w.in_cnt);
    } else if (k <= 32) {
        smooth_row_kernel<32><<<row_blocks, kThreads, 0, st>>>(idx, dist, n, k, KP, w.mean_all, w.rho, w.sigma,
                                                               w.scol, w.sw);
        count_group_kernel<32><<<g32_blocks, kThreads, 0, st>>>(n, KP, w.scol, w.sw, w.gv, w.tslot, w.own_cnt,
                                                                w.in_cnt);
    } else {
        smooth_warp_kernel<<<(unsigned)ceil_div(n, kWarpRows), kWarpRows * 32, 0, st>>>(
            idx, dist, n, k, w.mean_all, w.rho, w.sigma, w.scol, w.sw);
        count_kernel<<<row_blocks, kThreads, 0, st>>>(n, k, w.scol, w.sw, w.gv, w.own_cnt, w.in_cnt);
    }
    const int64_t nb = ceil_div(n, kScanTile);
    scan_local_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(n, w.own_cnt, w.in_cnt, indptr, w.scan_part);
    scan_part_kernel<<<1, 1024, 0, st>>>(nb, w.scan_part, n, indptr);
    scan_add_kernel<<<(unsigned)ceil_div(n, kScanThreads), kScanThreads, 0, st>>>(n, w.scan_part, indptr);
    return cudaGetLastError();
}

cudaError_t launch_conn_fill(int64_t n, int k, const int64_t *indptr, int32_t *indices,
                             float *data, int64_t cap, const ConnWork &w, cudaStream_t st) {
    const unsigned row_blocks = (unsigned)ceil_div(n, kThreads);
    const int KP = conn_stride(k);
    if (k <= 16) {
        fill_group_kernel<16><<<(unsigned)ceil_div(n, kThreads / 16), kThreads, 0, st>>>(
            n, KP, indptr, w.scol, w.gv, w.own_cnt, w.tslot, indices, data, cap, w.status);
    } else if (k <= 32) {
        fill_group_kernel<32><<<(unsigned)ceil_div(n, kThreads / 32), kThreads, 0, st>>>(
            n, KP, indptr, w.scol, w.gv, w.own_cnt, w.tslot, indices, data, cap, w.status);
    } else {
        fill_kernel<<<row_blocks, kThreads, 0, st>>>(n, k, indptr, w.scol, w.gv, w.own_cnt, w.cursor,
                                                     indices, data, cap, w.status);
    }
    sort_short_rows_kernel<<<row_blocks, kThreads, 0, st>>>(n, indptr, w.in_cnt, indices, data, cap, w.mid_rows,
                                                            w.mid_count, w.long_rows, w.long_count);
    sort_mid_rows_kernel<<<sm_count() * 4, kSortWarps * 32, 0, st>>>(indptr, indices, data, w.mid_rows,
                                                                    w.mid_count);
    sort_long_rows_kernel<<<sm_count() * 2, 1024, 0, st>>>(indptr, indices, data, w.long_rows,
                                                          w.long_count);
    return cudaGetLastError();
}

}  // namespace rsc
