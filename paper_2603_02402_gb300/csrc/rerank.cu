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
#include "warp_sort.cuh"

namespace rsc {

namespace {

constexpr int kWarps = 16;   // queries per block: neighbouring queries share candidate rows in L1

// Warp per query; E = (candidate slots rounded up to a power of two) / 32
// (key, id) pairs per lane, element v = e * 32 + lane.  The candidates are
// scored, then sorted ascending by (key, id) with a bitonic network held in
// registers: strides >= 32 compare a lane's own elements, smaller strides
// exchange with lane ^ stride by shuffles.
template <int E>
__global__ void __launch_bounds__(kWarps * 32)
rerank_kernel(const float *__restrict__ R, int64_t rs, int64_t n, int d, int metric, int w4,
              const int32_t *__restrict__ cand, int KC, int C, int k, const int32_t *__restrict__ perm,
              bool r_by_pos, int32_t *__restrict__ idx, float *__restrict__ dist) {
    __shared__ __align__(16) float xq_s[kWarps][68];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xq = xq_s[warp];   // query row (d <= 63 for cosine, so its flag fits) or d <= 64

    const int64_t q = (int64_t)blockIdx.x * kWarps + warp;   // position in the candidate lists
    if (q >= n) return;
    const int64_t qo = perm ? (int64_t)perm[q] : q;            // original row
    const int64_t qr = r_by_pos ? q : qo;                      // its row in R

    const bool cosine = metric == RSC_COSINE;
    const int width = cosine ? d + 1 : d;
    for (int t = lane; t < width; t += 32) xq[t] = R[qr * rs + t];
    __syncwarp();
    const bool fq = cosine && xq[d] != 0.f;

    float key[E];
    int id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = e * 32 + lane;
        key[e] = INFINITY;
        id[e] = INT_MAX;
        if (c < C) {
            const int s = c / KC, slot = c - s * KC;
            const int32_t jp = cand[((int64_t)s * n + q) * KC + slot];
            if (jp >= 0 && (int64_t)jp < n) {   // ids outside [0, n) (an aborted search) are skipped
                const int32_t j = perm ? perm[jp] : jp;                    // original id
                const float *yr = R + (int64_t)(r_by_pos ? jp : j) * rs;
                float acc = row_dist2(xq, yr, d, w4);
                if (cosine) {
                    const bool fy = __ldg(yr + d) != 0.f;
                    if (fq || fy) acc = (fq && fy) ? 0.f : 2.f;
                }
                key[e] = acc;
                id[e] = j;
            }
        }
    }

    warp_sort_pairs<E>(key, id);

#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = e * 32 + lane;
        if (c < k) {
            const bool valid = id[e] != INT_MAX;
            idx[qo * k + c] = valid ? id[e] : -1;
            dist[qo * k + c] = valid ? (cosine ? 0.5f * key[e] : sqrtf(key[e])) : INFINITY;
        }
    }
}

// dst row i <- src row perm[i] (width floats, zero-padded to dst_stride, a
// multiple of 4 with a 16-byte aligned dst); 16 lanes per row, a float4 store
// per lane and step.
__global__ void gather_rows_kernel(const float *__restrict__ src, int64_t src_stride, int64_t n, int width,
                                   const int32_t *__restrict__ perm, float *__restrict__ dst, int64_t dst_stride) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int l = threadIdx.x & 15;
    if (i >= n) return;
    const float *s = src + (int64_t)perm[i] * src_stride;
    float4 *o = reinterpret_cast<float4 *>(dst + i * dst_stride);
    for (int f = l; 4 * f < dst_stride; f += 16) {
        const int t = 4 * f;
        o[f] = make_float4(t < width ? s[t] : 0.f, t + 1 < width ? s[t + 1] : 0.f, t + 2 < width ? s[t + 2] : 0.f,
                           t + 3 < width ? s[t + 3] : 0.f);
    }
}

}  // namespace

cudaError_t launch_gather_rows(const float *src, int64_t src_stride, int64_t n, int width, const int32_t *perm,
                               float *dst, int64_t dst_stride, cudaStream_t st) {
    if (dst_stride % 4 != 0 || reinterpret_cast<uintptr_t>(dst) % 16 != 0) return cudaErrorInvalidValue;
    gather_rows_kernel<<<(unsigned)ceil_div(n * 16, 256), 256, 0, st>>>(src, src_stride, n, width, perm, dst,
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
    const unsigned blocks = (unsigned)ceil_div(n, kWarps);
    // vector loads when every row starts on a 16-byte boundary
    const int width = metric == RSC_COSINE ? d + 1 : d;
    const bool vec = rs % 4 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0 && width <= 64;
    const int w4 = vec ? (width + 3) / 4 : 0;
#define RSC_RR(e)                                                                                                   \
    case 32 * e:                                                                                                    \
        rerank_kernel<e><<<blocks, kWarps * 32, 0, st>>>(R, rs, n, d, metric, w4, cand, KC, C, k, perm, r_by_pos, \
                                                         idx, dist);                                                \
        break
    switch (C2) {
        RSC_RR(1); RSC_RR(2); RSC_RR(4); RSC_RR(8); RSC_RR(16); RSC_RR(32);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_RR
    return cudaGetLastError();
}

}  // namespace rsc
