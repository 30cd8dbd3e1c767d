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
// Every directed edge i -> j (weight a) is delivered to row j, so no pass
// reads another row's kNN list:
//   smooth  thread per row (k <= 32) or warp per row: rho, sigma (the
//           bisection is arithmetic; the bucket slots' atomics are issued
//           before it, so their latency hides behind it), the directed
//           weights, every edge pushed to its target's bucket of B slots (the
//           scatter-add with atomics of the paper's aggregation kernels,
//           Methods, "Custom GPU kernels"; pushes past B are flagged in a
//           per-row bit mask), the row's non-zero own entries sorted by column
//   match   G lanes per row: a bucket entry whose source is in the row's own
//           list is the reverse of a mutual edge: its weight b turns the own
//           value a into a + b - ab, and the entry leaves the bucket; the
//           other entries are compacted; flagged pushes are matched against
//           their target's own list by the source row (rare: in-degree > B)
//   scan    row pointers from own + bucket + flagged counts; the mean of all
//           distances and the floor of the rows without a non-zero distance
//   emit    per row: bucket entries ranked by counting, own and bucket
//           entries placed by rank (own entry x at x + #bucket entries below
//           it, bucket entry q at its rank + #own entries below it), so the
//           row is written in order; flagged entries go after their target's
//           bucket entries, and such rows are queued
//   sort    queued rows sorted whole (a warp in shared memory up to 512
//           entries, a block beyond)
#include <limits.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

constexpr int kThreads = 256;
constexpr int kBucket = 64;   // bucket slots per row (pushes merged in registers)
constexpr float kTol = 1e-5f;
constexpr int kIters = 64;
constexpr float kFloor = 1e-3f;

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

// Directed weight of an entry at distance d of a row with (rho, sigma); the
// self entry and empty slots are handled by the callers.  Every pass that
// needs a directed weight calls this, so all copies of a weight are the same
// bits.
__device__ __forceinline__ float directed_weight(float d, float rho, float sig) {
    const float g = d - rho;
    if (g <= 0.f || sig == 0.f) return 1.f;
    return expf(-(g / sig));
}

__device__ __forceinline__ float fuzzy_union(float a, float b) {
    // a + b - a*b, rounded the same way whichever endpoint computes it
    return __fsub_rn(__fadd_rn(a, b), __fmul_rn(a, b));
}

// Ascending bitonic sort of (key, val) pairs held E per lane across a group
// of G lanes; element x = e * G + l (l = lane in the group).  Strides of G
// and above compare registers of one lane, smaller strides exchange with the
// lane l ^ stride.  Keys are unique except the INT_MAX pads.
template <int G, int E>
__device__ __forceinline__ void group_bitonic(int (&key)[E], float (&val)[E], int l) {
    constexpr int N = G * E;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= G) {
                const int es = stride / G;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = e ^ es;
                    if (p > e) {
                        const bool asc = ((e * G + l) & size) == 0;
                        if ((key[e] > key[p]) == asc) {
                            const int tk = key[e];
                            key[e] = key[p];
                            key[p] = tk;
                            const float tv = val[e];
                            val[e] = val[p];
                            val[p] = tv;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pk = __shfl_xor_sync(0xffffffffu, key[e], stride);
                    const float pv = __shfl_xor_sync(0xffffffffu, val[e], stride);
                    const bool asc = ((e * G + l) & size) == 0;
                    const bool lower = (l & stride) == 0;
                    const bool take = (lower == asc) ? (pk < key[e]) : (pk > key[e]);
                    if (take) {
                        key[e] = pk;
                        val[e] = pv;
                    }
                }
            }
        }
    }
}

// Number of entries below x in the ascending array s[0 .. N) (N a power of
// two, INT_MAX pads at the end).
template <int N>
__device__ __forceinline__ int count_below(const int *s, int x) {
    int p = 0;
#pragma unroll
    for (int step = N / 2; step >= 1; step >>= 1)
        if (s[p + step - 1] < x) p += step;
    return p + (s[p] < x ? 1 : 0);
}

// ---------------------------------------------------------------- smooth

// 2^x by the ex2.approx.ftz.f32 instruction (PTX ISA; relative error about
// 2^-22, subnormal results flushed to 0, which no sum below can notice).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bisection of one row on g[c] = d_c - rho (entries at or past k are +inf
// and contribute 2^-inf = 0).  exp(-g / sigma) is evaluated as
// 2^(g * (-log2(e) / sigma)) with one reciprocal per step; the terms are
// summed pairwise (a balanced tree: rounding error grows with the tree depth,
// 4 levels for 15 terms, not with the number of terms).
template <int KM>
__device__ __forceinline__ float bisect_sigma(const float (&g)[KM], float target) {
    constexpr float kNegLog2e = -1.4426950408889634f;
    float lo = 0.f, hi = INFINITY, mid = 1.f;
    for (int it = 0; it < kIters; ++it) {
        const float sc = kNegLog2e * __frcp_rn(mid);
        float t[KM];
        t[0] = 0.f;
#pragma unroll
        for (int c = 1; c < KM; ++c) t[c] = (g[c] > 0.f) ? fast_exp2(g[c] * sc) : 1.f;
#pragma unroll
        for (int w = 1; w < KM; w <<= 1) {
#pragma unroll
            for (int c = 0; c + w < KM; c += 2 * w) t[c] += t[c + w];
        }
        const float psum = t[0];
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
    return mid;
}

// Thread per row, k <= KM (16 or 32).  Rows without a non-zero distance get
// the unfloored bisection result here and the global-mean floor in the scan
// pass; their weights are all 1 and do not depend on sigma.
template <int KM>
__global__ void __launch_bounds__(kThreads)
smooth_row_kernel(const float *__restrict__ dist, int64_t n, int k, float2 *__restrict__ rs,
                  float *__restrict__ rho_out, float *__restrict__ sigma_out, float *__restrict__ part_sum,
                  int32_t *__restrict__ rho0_rows, int32_t *__restrict__ rho0_count) {
    __shared__ float red[kThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float row_sum = 0.f;
    if (i < n) {
        const float *dr = dist + i * k;
        float dd[KM];
#pragma unroll
        for (int c = 0; c < KM; ++c) dd[c] = (c < k) ? dr[c] : 0.f;
        float r = 0.f;
        bool found = false;
#pragma unroll
        for (int c = 0; c < KM; ++c) {
            if (c < k && !found && dd[c] > 0.f) {
                r = dd[c];
                found = true;
            }
        }
#pragma unroll
        for (int c = 0; c < KM; ++c) row_sum += dd[c];
        float g[KM];
#pragma unroll
        for (int c = 0; c < KM; ++c) g[c] = (c < k) ? dd[c] - r : INFINITY;
        const float mid = bisect_sigma<KM>(g, log2f((float)k));
        float sig = mid;
        if (r > 0.f) {
            const float floor_v = kFloor * (row_sum / (float)k);
            if (sig < floor_v) sig = floor_v;
        } else {
            rho0_rows[atomicAdd(rho0_count, 1)] = (int32_t)i;
        }
        rs[i] = make_float2(r, sig);
        if (rho_out) rho_out[i] = r;
        if (sigma_out) sigma_out[i] = sig;
    }
    const float b = block_sum(row_sum, red);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = b;
}

// G lanes per row (k <= G), lane c holding entry c: the directed weight;
// every valid edge takes a bucket slot of its target (entries with weight 0
// fill their slot and are dropped by the match pass); pushes past B with a
// non-zero weight set bit c of ovf[i]; the non-zero own entries sorted by
// column across the group into ocol / og.  Few registers per lane, so many
// rows' atomics are in flight at once.
template <int G>
__global__ void __launch_bounds__(kThreads)
push_group_kernel(const int32_t *__restrict__ idx, const float *__restrict__ dist, int64_t n, int k, int KP, int B,
                  const float2 *__restrict__ rs, int32_t *__restrict__ in_cnt, int2 *__restrict__ bucket,
                  uint32_t *__restrict__ ovf, int32_t *__restrict__ ocol, float *__restrict__ og,
                  int32_t *__restrict__ own_cnt) {
    const int lane = threadIdx.x & 31, l = lane & (G - 1), base = lane & ~(G - 1);
    const unsigned gbits = (G == 32) ? 0xffffffffu : ((1u << G) - 1);
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / G) + lane / G;
    const bool row_ok = i < n;
    const int me = (int)i;
    int j = -1;
    float d = 0.f;
    if (row_ok && l < k) {
        const int32_t jj = idx[i * k + l];
        d = dist[i * k + l];
        if (jj >= 0 && (int64_t)jj < n && jj != me) j = jj;
    }
    const int slot = (j >= 0) ? atomicAdd(in_cnt + j, 1) : 0;
    float a = 0.f;
    if (j >= 0) {
        const float2 ri = rs[i];
        a = directed_weight(d, ri.x, ri.y);
    }
    bool spill = false;
    if (j >= 0) {
        if (slot < B) bucket[(int64_t)j * B + slot] = make_int2(me, __float_as_int(a));
        else spill = a != 0.f;
    }
    int key[1] = {(j >= 0 && a != 0.f) ? j : INT_MAX};
    float val[1] = {a};
    const unsigned own = (__ballot_sync(0xffffffffu, key[0] != INT_MAX) >> base) & gbits;
    const unsigned sp = (__ballot_sync(0xffffffffu, spill) >> base) & gbits;
    group_bitonic<G, 1>(key, val, l);
    if (row_ok) {
        if (l < KP) {
            ocol[i * KP + l] = key[0];
            og[i * KP + l] = val[0];
        }
        if (l == 0) {
            own_cnt[i] = __popc(own);
            ovf[i] = sp;
        }
    }
}

// Warp per row, 32 < k <= 32 E (entry c = lane + 32 e).  Flag bit of entry
// c: bit lane of ovf[i * E + e]; own entries sorted across the warp into
// ocol / og rows of KP = 32 E.
constexpr int kWarpRows = 4;

template <int E>
__global__ void __launch_bounds__(kWarpRows * 32)
smooth_push_warp_kernel(const int32_t *__restrict__ idx, const float *__restrict__ dist, int64_t n, int k, int KP,
                        int B, float2 *__restrict__ rs, float *__restrict__ rho_out, float *__restrict__ sigma_out,
                        float *__restrict__ part_sum, int32_t *__restrict__ rho0_rows,
                        int32_t *__restrict__ rho0_count, int32_t *__restrict__ in_cnt, int2 *__restrict__ bucket,
                        uint32_t *__restrict__ ovf, int32_t *__restrict__ ocol, float *__restrict__ og,
                        int32_t *__restrict__ own_cnt) {
    __shared__ float red[kWarpRows * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarpRows + warp;
    float rs_sum = 0.f;
    if (i < n) {   // uniform within the warp
        const int me = (int)i;
        float dd[E];
        int col[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = lane + 32 * e;
            dd[e] = 0.f;
            col[e] = -1;
            if (c < k) {
                const int32_t j = idx[i * k + c];
                dd[e] = dist[i * k + c];
                if (j >= 0 && (int64_t)j < n && j != me) col[e] = j;
            }
        }
        int slot[E];
#pragma unroll
        for (int e = 0; e < E; ++e) slot[e] = (col[e] >= 0) ? atomicAdd(in_cnt + col[e], 1) : 0;
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
            if (mid == prev) break;
        }
        float sum = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) sum += dd[e];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        float sig = mid;
        if (r > 0.f) {
            const float floor_v = kFloor * (sum / (float)k);
            if (sig < floor_v) sig = floor_v;
        } else if (lane == 0) {
            rho0_rows[atomicAdd(rho0_count, 1)] = me;
        }
        if (lane == 0) {
            rs[i] = make_float2(r, sig);
            if (rho_out) rho_out[i] = r;
            if (sigma_out) sigma_out[i] = sig;
            rs_sum = sum;
        }
        int key[E];
        float a[E];
        int cnt = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            a[e] = 0.f;
            bool spill = false;
            if (col[e] >= 0) {
                a[e] = directed_weight(dd[e], r, sig);
                if (slot[e] < B) bucket[(int64_t)col[e] * B + slot[e]] = make_int2(me, __float_as_int(a[e]));
                else spill = a[e] != 0.f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, spill);
            if (lane == 0) ovf[i * E + e] = m;
            key[e] = (col[e] >= 0 && a[e] != 0.f) ? col[e] : INT_MAX;
            cnt += __popc(__ballot_sync(0xffffffffu, key[e] != INT_MAX));
        }
        group_bitonic<32, E>(key, a, lane);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            ocol[i * KP + e * 32 + lane] = key[e];
            og[i * KP + e * 32 + lane] = a[e];
        }
        if (lane == 0) own_cnt[i] = cnt;
    }
    const float b = block_sum(rs_sum, red);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = b;
}

// ----------------------------------------------------------------- match

// G lanes per row, own entries E per lane (x = e * G + l), bucket entries
// NB per lane (q = e * G + l, B = NB G).  A bucket entry whose source is an
// own entry is the reverse of a mutual edge: the own value becomes
// a + b - ab and the entry is dropped; entries with weight 0 are dropped;
// the rest are compacted to the front of the bucket (in_kept of them).  The
// row's flagged pushes (its edges that found the target's bucket full) are
// looked up in the target's own list: a mutual one updates the target's own
// value, the others count toward the target's row (extra) and keep their
// flag for the emit pass.
template <int G, int E, int NB>
__global__ void __launch_bounds__(kThreads)
match_kernel(const int32_t *__restrict__ idx, const float *__restrict__ dist, int64_t n, int k, int KP, int B,
             int MW, const float2 *__restrict__ rs, const int32_t *__restrict__ ocol, float *__restrict__ og,
             const int32_t *__restrict__ own_cnt, const int32_t *__restrict__ in_cnt, int2 *__restrict__ bucket,
             uint32_t *__restrict__ ovf, int32_t *__restrict__ in_kept, int32_t *__restrict__ extra) {
    constexpr int GPW = 32 / G;
    __shared__ int s_own[kThreads / 32][GPW][G * E];
    __shared__ float s_hit[kThreads / 32][GPW][G * E];
    const int lane = threadIdx.x & 31, l = lane & (G - 1), grp = lane / G, warp = threadIdx.x >> 5;
    const int base = grp * G;
    const unsigned gbits = (G == 32) ? 0xffffffffu : ((1u << G) - 1);
    const unsigned gmask = gbits << base;
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW + grp;
    const bool row_ok = i < n;
    int oc = 0, ic = 0;
    if (row_ok) {
        oc = own_cnt[i];
        ic = min(in_cnt[i], B);
    }
    const int32_t *orow = ocol + (size_t)(row_ok ? i : 0) * KP;
    float *grow = og + (size_t)(row_ok ? i : 0) * KP;
    int2 *brow = bucket + (size_t)(row_ok ? i : 0) * B;
    int *so = s_own[warp][grp];
    float *sh = s_hit[warp][grp];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = e * G + l;
        so[x] = (x < oc) ? orow[x] : INT_MAX;
        sh[x] = 0.f;
    }
    int src[NB];
    float wa[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        const int q = e * G + l;
        src[e] = INT_MAX;
        wa[e] = 0.f;
        if (q < ic) {
            const int2 t = brow[q];
            src[e] = t.x;
            wa[e] = __int_as_float(t.y);
        }
    }
    __syncwarp();
    bool kept[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        kept[e] = false;
        if (src[e] != INT_MAX) {
            const int p = count_below<G * E>(so, src[e]);
            if (p < oc && so[p] == src[e]) {
                if (wa[e] != 0.f) sh[p] = wa[e];
            } else {
                kept[e] = wa[e] != 0.f;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = e * G + l;
        if (x < oc && sh[x] != 0.f) grow[x] = fuzzy_union(grow[x], sh[x]);
    }
    const unsigned lt = (1u << l) - 1u;
    int run = 0;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        const unsigned m = (__ballot_sync(0xffffffffu, kept[e]) >> base) & gbits;
        if (kept[e]) brow[run + __popc(m & lt)] = make_int2(src[e], __float_as_int(wa[e]));
        run += __popc(m);
    }
    if (row_ok && l == 0) in_kept[i] = run;
    if (!row_ok) return;   // uniform within the group; no warp-wide step follows
    const int me = (int)i;
    for (int w = 0; w < MW; ++w) {
        const uint32_t m = ovf[i * MW + w];
        if (m == 0) continue;   // uniform within the group
        const int c = w * 32 + l;
        bool keep = false;
        if ((m >> l) & 1u) {
            const int32_t t = idx[i * k + c];
            const float2 ri = rs[i];
            const float a = directed_weight(dist[i * k + c], ri.x, ri.y);
            const int32_t *tr = ocol + (size_t)t * KP;
            int lo = 0, hi = own_cnt[t];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (tr[mid] < me) lo = mid + 1;
                else hi = mid;
            }
            if (lo < own_cnt[t] && tr[lo] == me) {
                float *gp = og + (size_t)t * KP + lo;
                *gp = fuzzy_union(*gp, a);
            } else {
                atomicAdd(extra + t, 1);
                keep = true;
            }
        }
        const unsigned km = (__ballot_sync(gmask, keep) >> base) & gbits;
        if (l == 0) ovf[i * MW + w] = km;
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

// Row lengths own + bucket + flagged -> offsets inside each tile of
// kScanTile rows (local) and the tiles' totals (part).
__global__ void __launch_bounds__(kScanThreads)
scan_local_kernel(int64_t n, const int32_t *__restrict__ own_cnt, const int32_t *__restrict__ in_kept,
                  const int32_t *__restrict__ extra, int64_t *__restrict__ local, int64_t *__restrict__ part) {
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const int64_t i = base + e;
        v[e] = (i < n) ? (int64_t)own_cnt[i] + (int64_t)in_kept[i] + (int64_t)extra[i] : 0;
        sum += v[e];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(sum, warp_sums, total);
#pragma unroll
    for (int e = 0; e < kScanItems; ++e) {
        const int64_t i = base + e;
        if (i < n) local[i] = run;
        run += v[e];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: exclusive scan of the tile totals (indptr[n] = nnz), then the
// mean of all distances from the smooth pass's partial sums and the floor
// 1e-3 * mean of the rows without a non-zero distance.
__global__ void __launch_bounds__(1024)
scan_part_kernel(int64_t nb, int64_t *__restrict__ part, int64_t n, int64_t *__restrict__ indptr,
                 const float *__restrict__ part_sum, int64_t n_sum, int64_t total_entries,
                 const int32_t *__restrict__ rho0_rows, const int32_t *__restrict__ rho0_count,
                 float2 *__restrict__ rs, float *__restrict__ sigma_out) {
    __shared__ int64_t warp_sums[32];
    __shared__ float red[1024];
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
    const int c0 = *rho0_count;
    if (c0 == 0) return;   // uniform
    float s = 0.f;
    for (int64_t b = threadIdx.x; b < n_sum; b += blockDim.x) s += part_sum[b];
    const float mean_all = block_sum(s, red) / (float)total_entries;
    const float floor_v = kFloor * mean_all;
    for (int r = threadIdx.x; r < c0; r += blockDim.x) {
        const int32_t i = rho0_rows[r];
        float2 v = rs[i];
        if (v.y < floor_v) v.y = floor_v;
        rs[i] = v;
        if (sigma_out) sigma_out[i] = v.y;
    }
}

// indptr[i] = local[i] + part[tile of i] (used when the CSR is not filled).
__global__ void __launch_bounds__(kScanThreads)
scan_add_kernel(int64_t n, const int64_t *__restrict__ local, const int64_t *__restrict__ part,
                int64_t *__restrict__ indptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) indptr[i] = local[i] + part[i / kScanTile];
}

// ------------------------------------------------------------------ emit

constexpr int kWarpSortMax = 512;
constexpr int kBlockSortMax = 4096;

// The host launches the fill only when the CSR capacity holds nnz, so every
// position is in range.
__device__ __forceinline__ void put(int32_t *indices, float *data, int64_t p, int c, float v) {
    indices[p] = c;
    data[p] = v;
}

// G lanes per row.  A row without flagged entries: its kept bucket entries
// (at most B = NB G, NB per lane) are ranked by counting (rank = entries with
// a smaller source), written to shared memory in order, and each own and
// bucket entry is placed at its rank in the union.  A row with flagged
// entries gets its own and bucket entries written unsorted and is queued for
// a whole-row sort; its flagged entries are placed by their source rows,
// after its bucket entries.
template <int G, int E, int NB>
__global__ void __launch_bounds__(kThreads)
emit_kernel(int64_t n, int k, int KP, int B, int MW, const int32_t *__restrict__ idx,
            const float *__restrict__ dist, const float2 *__restrict__ rs, const int32_t *__restrict__ ocol,
            const float *__restrict__ og, const int32_t *__restrict__ own_cnt, const int32_t *__restrict__ in_kept,
            const int32_t *__restrict__ extra, const int2 *__restrict__ bucket, const uint32_t *__restrict__ ovf,
            const int64_t *__restrict__ local, const int64_t *__restrict__ part, int64_t *__restrict__ indptr,
            int32_t *__restrict__ cursor, int32_t *__restrict__ indices, float *__restrict__ data, int64_t cap,
            int32_t *__restrict__ mid_rows, int32_t *__restrict__ mid_count, int32_t *__restrict__ long_rows,
            int32_t *__restrict__ long_count, unsigned int *status) {
    constexpr int GPW = 32 / G;   // rows per warp
    static_assert(NB >= 2, "the bucket holds at least the 2G entries a row merges in registers");
    __shared__ int s_own[kThreads / 32][GPW][G * E];
    __shared__ int s_in[kThreads / 32][GPW][2 * G];
    const int lane = threadIdx.x & 31, l = lane & (G - 1), grp = lane / G, warp = threadIdx.x >> 5;
    const int base = grp * G;
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW + grp;
    const bool row_ok = i < n;
    int64_t start = 0;
    int oc = 0, ic = 0, ex = 0;
    if (row_ok) {
        start = local[i] + part[i / kScanTile];
        oc = own_cnt[i];
        ic = in_kept[i];
        ex = extra[i];
        if (l == 0) indptr[i] = start;
    }
    const int32_t *orow = ocol + (size_t)(row_ok ? i : 0) * KP;
    const float *grow = og + (size_t)(row_ok ? i : 0) * KP;
    const int2 *brow = bucket + (size_t)(row_ok ? i : 0) * B;
    int col[E];
    float gv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = e * G + l;
        col[e] = (x < oc) ? orow[x] : INT_MAX;
        gv[e] = (x < oc) ? grow[x] : 0.f;
    }
    int src[NB];
    float wa[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) {
        const int q = e * G + l;
        src[e] = INT_MAX;
        wa[e] = 0.f;
        if (q < ic) {
            const int2 t = brow[q];
            src[e] = t.x;
            wa[e] = __int_as_float(t.y);
        }
    }
    // rows with flagged entries or more bucket entries than the merge's
    // 2G are written unsorted and queued
    const bool hub = ex > 0 || ic > 2 * G;
    if (hub) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = e * G + l;
            if (x < oc) put(indices, data, start + x, col[e], gv[e]);
        }
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            const int q = e * G + l;
            if (q < ic) put(indices, data, start + oc + q, src[e], wa[e]);
        }
        if (l == 0) {
            const int L = oc + ic + ex;
            if (L <= kWarpSortMax) mid_rows[atomicAdd(mid_count, 1)] = (int32_t)i;
            else long_rows[atomicAdd(long_count, 1)] = (int32_t)i;
        }
    }
    // ranks of the bucket entries (pads are INT_MAX and never below a key);
    // merged rows hold at most 2G of them, in src[0 .. 2)
    const int icmax = __reduce_max_sync(0xffffffffu, hub ? 0 : ic);
    int rk[NB];
#pragma unroll
    for (int e = 0; e < NB; ++e) rk[e] = 0;
    for (int t = 0; t < icmax; ++t) {
        const int v = __shfl_sync(0xffffffffu, t < G ? src[0] : src[1], base + (t & (G - 1)));
        rk[0] += v < src[0];
        rk[1] += v < src[1];
    }
    int *so = s_own[warp][grp];
    int *si = s_in[warp][grp];
#pragma unroll
    for (int e = 0; e < E; ++e) so[e * G + l] = col[e];
    // position p < ic holds the entry of rank p, p >= ic a pad (ranks are a
    // permutation of [0, ic): sources are distinct)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int q = e * G + l;
        si[(!hub && q < ic) ? rk[e] : q] = src[e];
    }
    __syncwarp();
    if (row_ok && !hub) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = e * G + l;
            if (x < oc) put(indices, data, start + x + count_below<2 * G>(si, col[e]), col[e], gv[e]);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = e * G + l;
            if (q < ic) put(indices, data, start + rk[e] + count_below<G * E>(so, src[e]), src[e], wa[e]);
        }
    }
    // this row's flagged edges go after the bucket entries of their targets
    if (row_ok) {
        for (int w = 0; w < MW; ++w) {
            const uint32_t m = ovf[i * MW + w];
            if (m == 0) continue;   // uniform within the group
            const int c = w * 32 + l;
            if ((m >> l) & 1u) {
                const int32_t t = idx[i * k + c];
                const float2 ri = rs[i];
                const float a = directed_weight(dist[i * k + c], ri.x, ri.y);
                const int slot = atomicAdd(cursor + t, 1);
                const int64_t p = local[t] + part[t / kScanTile] + own_cnt[t] + in_kept[t] + slot;
                put(indices, data, p, (int32_t)i, a);
            }
        }
    }
}

// ------------------------------------------------------------------ sort

constexpr int kSortWarps = 8;

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

// Warp per queued row of up to kWarpSortMax entries, in shared memory.
__global__ void __launch_bounds__(kSortWarps * 32)
sort_mid_rows_kernel(const int64_t *__restrict__ indptr, int32_t *__restrict__ indices, float *__restrict__ data,
                     int64_t cap, const int32_t *__restrict__ mid_rows, const int32_t *__restrict__ mid_count) {
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
        if (b + L > cap) continue;   // capacity error already recorded
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
                      float *__restrict__ data, int64_t cap, const int32_t *__restrict__ long_rows,
                      const int32_t *__restrict__ long_count) {
    __shared__ int s_col[kBlockSortMax];
    __shared__ float s_w[kBlockSortMax];
    const int cnt = *long_count;
    for (int r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = long_rows[r];
        const int64_t b = indptr[i];
        const int L = (int)(indptr[i + 1] - b);
        if (b + L > cap) continue;   // uniform: capacity error already recorded
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

template <int G, int E, int NB = kBucket / G>
void launch_match(const int32_t *idx, const float *dist, int64_t n, int k, const ConnShape &s, const ConnWork &w,
                  cudaStream_t st) {
    const unsigned blocks = (unsigned)ceil_div(n, kThreads / 32 * (32 / G));
    match_kernel<G, E, NB><<<blocks, kThreads, 0, st>>>(idx, dist, n, k, s.KP, s.B, s.MW, w.rs, w.ocol, w.og, w.own_cnt,
                                                    w.in_cnt, w.bucket, w.ovf, w.in_kept, w.extra);
}

template <int G, int E, int NB = kBucket / G>
void launch_emit(const int32_t *idx, const float *dist, int64_t n, int k, const ConnShape &s, int64_t *indptr,
                 int32_t *indices, float *data, int64_t cap, const ConnWork &w, cudaStream_t st) {
    const unsigned blocks = (unsigned)ceil_div(n, kThreads / 32 * (32 / G));
    emit_kernel<G, E, NB><<<blocks, kThreads, 0, st>>>(n, k, s.KP, s.B, s.MW, idx, dist, w.rs, w.ocol, w.og, w.own_cnt,
                                                   w.in_kept, w.extra, w.bucket, w.ovf, w.local, w.scan_part, indptr,
                                                   w.cursor, indices, data, cap, w.mid_rows, w.mid_count,
                                                   w.long_rows, w.long_count, w.status);
}

template <int E>
void launch_smooth_warp(const int32_t *idx, const float *dist, int64_t n, int k, const ConnShape &s, float *rho_out,
                        float *sigma_out, const ConnWork &w, unsigned blocks, cudaStream_t st) {
    smooth_push_warp_kernel<E><<<blocks, kWarpRows * 32, 0, st>>>(idx, dist, n, k, s.KP, s.B, w.rs, rho_out,
                                                                  sigma_out, w.part_sum, w.rho0_rows, w.rho0_count,
                                                                  w.in_cnt, w.bucket, w.ovf, w.ocol, w.og,
                                                                  w.own_cnt);
}

}  // namespace

ConnShape conn_shape(int k) {
    ConnShape s;
    s.G = (k <= 16) ? 16 : 32;
    s.E = (k <= 32) ? 1 : (k <= 64 ? 2 : (k <= 128 ? 4 : 8));
    s.KP = (k <= 32) ? (k + 3) / 4 * 4 : 32 * s.E;
    s.B = kBucket;
    s.MW = s.E;
    s.smooth_rows = (k <= 32) ? kThreads : kWarpRows;
    return s;
}

size_t conn_scan_blocks(int64_t n) { return (size_t)ceil_div(n, kScanTile); }

size_t conn_sum_blocks(int64_t n, int k) { return (size_t)ceil_div(n, conn_shape(k).smooth_rows); }

cudaError_t launch_conn_count(const int32_t *idx, const float *dist, int64_t n, int k, int64_t *indptr,
                              float *rho_out, float *sigma_out, const ConnWork &w, cudaStream_t st) {
    const ConnShape s = conn_shape(k);
    const unsigned sum_blocks = (unsigned)conn_sum_blocks(n, k);
    if (k <= 16) {
        smooth_row_kernel<16><<<sum_blocks, kThreads, 0, st>>>(dist, n, k, w.rs, rho_out, sigma_out, w.part_sum,
                                                                w.rho0_rows, w.rho0_count);
        push_group_kernel<16><<<(unsigned)ceil_div(n, kThreads / 16), kThreads, 0, st>>>(
            idx, dist, n, k, s.KP, s.B, w.rs, w.in_cnt, w.bucket, w.ovf, w.ocol, w.og, w.own_cnt);
    } else if (k <= 32) {
        smooth_row_kernel<32><<<sum_blocks, kThreads, 0, st>>>(dist, n, k, w.rs, rho_out, sigma_out, w.part_sum,
                                                                w.rho0_rows, w.rho0_count);
        push_group_kernel<32><<<(unsigned)ceil_div(n, kThreads / 32), kThreads, 0, st>>>(
            idx, dist, n, k, s.KP, s.B, w.rs, w.in_cnt, w.bucket, w.ovf, w.ocol, w.og, w.own_cnt);
    }
    else if (k <= 64) launch_smooth_warp<2>(idx, dist, n, k, s, rho_out, sigma_out, w, sum_blocks, st);
    else if (k <= 128) launch_smooth_warp<4>(idx, dist, n, k, s, rho_out, sigma_out, w, sum_blocks, st);
    else launch_smooth_warp<8>(idx, dist, n, k, s, rho_out, sigma_out, w, sum_blocks, st);
    if (k <= 16) launch_match<16, 1>(idx, dist, n, k, s, w, st);
    else if (k <= 32) launch_match<32, 1>(idx, dist, n, k, s, w, st);
    else if (k <= 64) launch_match<32, 2>(idx, dist, n, k, s, w, st);
    else if (k <= 128) launch_match<32, 4>(idx, dist, n, k, s, w, st);
    else launch_match<32, 8>(idx, dist, n, k, s, w, st);
    const int64_t nb = ceil_div(n, kScanTile);
    scan_local_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(n, w.own_cnt, w.in_kept, w.extra, w.local,
                                                             w.scan_part);
    scan_part_kernel<<<1, 1024, 0, st>>>(nb, w.scan_part, n, indptr, w.part_sum, (int64_t)sum_blocks,
                                         n * (int64_t)k, w.rho0_rows, w.rho0_count, w.rs, sigma_out);
    return cudaGetLastError();
}

cudaError_t launch_conn_indptr(int64_t n, int64_t *indptr, const ConnWork &w, cudaStream_t st) {
    scan_add_kernel<<<(unsigned)ceil_div(n, kScanThreads), kScanThreads, 0, st>>>(n, w.local, w.scan_part, indptr);
    return cudaGetLastError();
}

cudaError_t launch_conn_fill(const int32_t *idx, const float *dist, int64_t n, int k, int64_t *indptr,
                             int32_t *indices, float *data, int64_t cap, const ConnWork &w, cudaStream_t st) {
    const ConnShape s = conn_shape(k);
    if (k <= 16) launch_emit<16, 1>(idx, dist, n, k, s, indptr, indices, data, cap, w, st);
    else if (k <= 32) launch_emit<32, 1>(idx, dist, n, k, s, indptr, indices, data, cap, w, st);
    else if (k <= 64) launch_emit<32, 2>(idx, dist, n, k, s, indptr, indices, data, cap, w, st);
    else if (k <= 128) launch_emit<32, 4>(idx, dist, n, k, s, indptr, indices, data, cap, w, st);
    else launch_emit<32, 8>(idx, dist, n, k, s, indptr, indices, data, cap, w, st);
    sort_mid_rows_kernel<<<sm_count() * 4, kSortWarps * 32, 0, st>>>(indptr, indices, data, cap, w.mid_rows,
                                                                    w.mid_count);
    sort_long_rows_kernel<<<sm_count() * 2, 1024, 0, st>>>(indptr, indices, data, cap, w.long_rows, w.long_count);
    return cudaGetLastError();
}

}  // namespace rsc
