// Exact FP32 re-rank of the candidate lists.
//
// Candidate selection (FP32 expansion form or BF16 tensor cores) only has to
// bring the true k nearest into each query's candidate set; this pass
// re-scores every candidate by direct difference, sum_t (x_t - y_t)^2 in FP32
// (no cancellation against |x|^2 + |y|^2), and orders by (distance, id), the
// exact-kNN definition with ties broken by index.  Cosine rows arrive
// normalised, so 1 - cos = |x^ - y^|^2 / 2 (paper, Methods, "Custom GPU
// kernels", defines both distances).
#include <math.h>
#include <limits.h>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

constexpr int kWarps = 4;

__device__ __forceinline__ bool pair_gt(float ka, int ia, float kb, int ib) {
    return ka > kb || (ka == kb && ia > ib);
}

// Squared distance sum_t (xq_t - y_t)^2 for t < d, accumulated in t order
// (the same rounding whichever loader runs).  W4 > 0: the row is 16-byte
// aligned and its first 4 * W4 floats are read as W4 independent float4
// loads up front; W4 == 0: scalar loads.
template <int W4>
__device__ __forceinline__ float row_dist2(const float *xq, const float *__restrict__ yr, int d) {
    float acc = 0.f;
    if constexpr (W4 > 0) {
        float y[4 * W4];
        const float4 *y4 = reinterpret_cast<const float4 *>(yr);
#pragma unroll
        for (int u = 0; u < W4; ++u) {
            const float4 v = __ldg(y4 + u);
            y[4 * u] = v.x;
            y[4 * u + 1] = v.y;
            y[4 * u + 2] = v.z;
            y[4 * u + 3] = v.w;
        }
#pragma unroll
        for (int t = 0; t < 4 * W4; ++t) {
            if (t < d) {
                const float diff = xq[t] - y[t];
                acc = fmaf(diff, diff, acc);
            }
        }
    } else {
        for (int t = 0; t < d; ++t) {
            const float diff = xq[t] - __ldg(yr + t);
            acc = fmaf(diff, diff, acc);
        }
    }
    return acc;
}

template <int W4>
__global__ void __launch_bounds__(kWarps * 32)
rerank_kernel(const float *__restrict__ R, int64_t rs, int64_t n, int d, int metric,
              const int32_t *__restrict__ cand, int KC, int C, int C2, int k, const int32_t *__restrict__ perm,
              bool r_by_pos, int32_t *__restrict__ idx, float *__restrict__ dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int XQ = 65;   // query row (d <= 63 for cosine, so its flag fits) or d <= 64
    float *xq = reinterpret_cast<float *>(smem) + warp * XQ;
    float *skey = reinterpret_cast<float *>(smem) + kWarps * XQ + warp * C2;
    int *sid = reinterpret_cast<int *>(reinterpret_cast<float *>(smem) + kWarps * XQ + kWarps * C2) + warp * C2;

    const int64_t q = (int64_t)blockIdx.x * kWarps + warp;   // position in the candidate lists
    if (q >= n) return;
    const int64_t qo = perm ? (int64_t)perm[q] : q;            // original row
    const int64_t qr = r_by_pos ? q : qo;                      // its row in R

    const bool cosine = metric == RSC_COSINE;
    const int width = cosine ? d + 1 : d;
    for (int t = lane; t < width; t += 32) xq[t] = R[qr * rs + t];
    __syncwarp();
    const bool fq = cosine && xq[d] != 0.f;

    for (int c = lane; c < C2; c += 32) {
        float key = INFINITY;
        int id = INT_MAX;
        if (c < C) {
            const int s = c / KC, slot = c - s * KC;
            const int32_t jp = cand[((int64_t)s * n + q) * KC + slot];
            if (jp >= 0) {
                const int32_t j = perm ? perm[jp] : jp;                    // original id
                const float *yr = R + (int64_t)(r_by_pos ? jp : j) * rs;
                float acc = row_dist2<W4>(xq, yr, d);
                if (cosine) {
                    const bool fy = __ldg(yr + d) != 0.f;
                    if (fq || fy) acc = (fq && fy) ? 0.f : 2.f;
                }
                key = acc;
                id = j;
            }
        }
        skey[c] = key;
        sid[c] = id;
    }
    __syncwarp();

    // bitonic sort of C2 (a power of two) pairs, ascending by (key, id)
    for (int size = 2; size <= C2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < C2 / 2; i += 32) {
                const int lo = (i / stride) * 2 * stride + (i % stride);
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const float ka = skey[lo], kb = skey[hi];
                const int ia = sid[lo], ib = sid[hi];
                const bool swap = asc ? pair_gt(ka, ia, kb, ib) : pair_gt(kb, ib, ka, ia);
                if (swap) {
                    skey[lo] = kb;
                    skey[hi] = ka;
                    sid[lo] = ib;
                    sid[hi] = ia;
                }
            }
            __syncwarp();
        }
    }

    for (int c = lane; c < k; c += 32) {
        const int id = sid[c];
        const float key = skey[c];
        const bool valid = id != INT_MAX;
        idx[qo * k + c] = valid ? id : -1;
        dist[qo * k + c] = valid ? (cosine ? 0.5f * key : sqrtf(key)) : INFINITY;
    }
}

// dst row i <- src row perm[i] (width floats); warp per row.
__global__ void gather_rows_kernel(const float *__restrict__ src, int64_t src_stride, int64_t n, int width,
                                   const int32_t *__restrict__ perm, float *__restrict__ dst, int64_t dst_stride) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const float *s = src + (int64_t)perm[i] * src_stride;
    float *o = dst + i * dst_stride;
    for (int t = lane; t < dst_stride; t += 32) o[t] = t < width ? s[t] : 0.f;
}

}  // namespace

cudaError_t launch_gather_rows(const float *src, int64_t src_stride, int64_t n, int width, const int32_t *perm,
                               float *dst, int64_t dst_stride, cudaStream_t st) {
    gather_rows_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, st>>>(src, src_stride, n, width, perm, dst,
                                                                      dst_stride);
    return cudaGetLastError();
}

cudaError_t launch_rerank(const float *R, int64_t rs, int64_t n, int d, int metric,
                          const int32_t *cand, int KC, int splits, int k, const int32_t *perm, bool r_by_pos,
                          int32_t *idx, float *dist, cudaStream_t st) {
    const int C = KC * splits;
    int C2 = 32;
    while (C2 < C) C2 <<= 1;
    if (C2 > 1024 || k > C) return cudaErrorInvalidValue;
    constexpr int XQ = 65;
    const size_t smem = sizeof(float) * kWarps * XQ + (sizeof(float) + sizeof(int)) * kWarps * C2;
    const unsigned blocks = (unsigned)ceil_div(n, kWarps);
    // vector loads when every row starts on a 16-byte boundary
    const int width = metric == RSC_COSINE ? d + 1 : d;
    const bool vec = rs % 4 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0 && width <= 64;
    const int W4 = vec ? (width + 3) / 4 : 0;
#define RSC_RR(w4)                                                                                              \
    case w4:                                                                                                    \
        rerank_kernel<w4><<<blocks, kWarps * 32, smem, st>>>(R, rs, n, d, metric, cand, KC, C, C2, k, perm,     \
                                                             r_by_pos, idx, dist);                              \
        break
    switch (W4) {
        RSC_RR(0); RSC_RR(1); RSC_RR(2); RSC_RR(3); RSC_RR(4); RSC_RR(5); RSC_RR(6); RSC_RR(7); RSC_RR(8);
        RSC_RR(9); RSC_RR(10); RSC_RR(11); RSC_RR(12); RSC_RR(13); RSC_RR(14); RSC_RR(15); RSC_RR(16);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_RR
    return cudaGetLastError();
}

}  // namespace rsc
