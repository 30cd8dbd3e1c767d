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

__global__ void __launch_bounds__(kWarps * 32)
rerank_kernel(const float *__restrict__ R, int64_t rs, int64_t n, int d, int metric,
              const int32_t *__restrict__ cand, int KC, int C, int C2, int k, const int32_t *__restrict__ perm,
              int32_t *__restrict__ idx, float *__restrict__ dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int XQ = 65;   // query row (d <= 63 for cosine, so its flag fits) or d <= 64
    float *xq = reinterpret_cast<float *>(smem) + warp * XQ;
    float *skey = reinterpret_cast<float *>(smem) + kWarps * XQ + warp * C2;
    int *sid = reinterpret_cast<int *>(reinterpret_cast<float *>(smem) + kWarps * XQ + kWarps * C2) + warp * C2;

    const int64_t q = (int64_t)blockIdx.x * kWarps + warp;   // position in the candidate lists
    if (q >= n) return;
    const int64_t qo = perm ? (int64_t)perm[q] : q;            // original row

    const bool cosine = metric == RSC_COSINE;
    const int width = cosine ? d + 1 : d;
    for (int t = lane; t < width; t += 32) xq[t] = R[qo * rs + t];
    __syncwarp();
    const bool fq = cosine && xq[d] != 0.f;

    for (int c = lane; c < C2; c += 32) {
        float key = INFINITY;
        int id = INT_MAX;
        if (c < C) {
            const int s = c / KC, slot = c - s * KC;
            int32_t j = cand[((int64_t)s * n + q) * KC + slot];
            if (j >= 0) {
                if (perm) j = perm[j];
                const float *yr = R + (int64_t)j * rs;
                float acc = 0.f;
                for (int t = 0; t < d; ++t) {
                    const float diff = xq[t] - __ldg(yr + t);
                    acc = fmaf(diff, diff, acc);
                }
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

}  // namespace

cudaError_t launch_rerank(const float *R, int64_t rs, int64_t n, int d, int metric,
                          const int32_t *cand, int KC, int splits, int k, const int32_t *perm, int32_t *idx,
                          float *dist, cudaStream_t st) {
    const int C = KC * splits;
    int C2 = 32;
    while (C2 < C) C2 <<= 1;
    if (C2 > 1024 || k > C) return cudaErrorInvalidValue;
    constexpr int XQ = 65;
    const size_t smem = sizeof(float) * kWarps * XQ + (sizeof(float) + sizeof(int)) * kWarps * C2;
    const unsigned blocks = (unsigned)ceil_div(n, kWarps);
    rerank_kernel<<<blocks, kWarps * 32, smem, st>>>(R, rs, n, d, metric, cand, KC, C, C2, k, perm, idx, dist);
    return cudaGetLastError();
}

}  // namespace rsc
