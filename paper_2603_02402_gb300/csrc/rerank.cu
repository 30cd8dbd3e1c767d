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

// Warp per query, 8 lanes per candidate row.  In step g, lanes 8 r + s
// (r < 4, s < 8) score candidate 4 g + r of the current 32: lane s takes
// components 4 s .. 4 s + 3 and 32 + 4 s .. 32 + 4 s + 3 (two 16-byte loads
// when rows start on 16-byte boundaries, else scalar loads; the same sums
// either way), an FMA chain over its eight, and three xor shuffles add the
// eight partial sums; candidate c's sum then goes to lane c % 32.  One load
// instruction of the warp touches 4 candidate rows instead of 32 (a lane per
// row): the gathers are bound by the L1's line lookups, not by bytes.
// E = (candidate slots rounded up to a power of two) / 32 (key, id) pairs per
// lane, element v = e * 32 + lane, sorted ascending by (key, id) with a
// bitonic network held in registers.  Up to 64 candidates fit in 32 registers
// a thread, so four blocks (all 64 warps) stay resident to hide the gathers'
// latency.
template <int E>
__global__ void __launch_bounds__(kWarps * 32, E <= 2 ? 4 : 1)
rerank_kernel(const float *__restrict__ R, int64_t rs, int64_t n, int d, int metric, bool vec,
              const int32_t *__restrict__ cand, int KC, int C, int k, const int32_t *__restrict__ perm,
              bool r_by_pos, int32_t *__restrict__ idx, float *__restrict__ dist) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane >> 3, s = lane & 7;

    const int64_t q = (int64_t)blockIdx.x * kWarps + warp;   // position in the candidate lists
    if (q >= n) return;                                        // warp-uniform
    const int64_t qo = perm ? (int64_t)perm[q] : q;            // original row
    const int64_t qr = r_by_pos ? q : qo;                      // its row in R
    const bool cosine = metric == RSC_COSINE;

    // this lane's components of a row.  Loads stop at the last 4-aligned piece
    // holding a component below d; the rest of that piece is zero padding
    // except the cosine rows' flag at column d, which is cleared.
    auto load8 = [&](const float *row, float (&v)[8]) {
        if (vec) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
            const float4 a = (4 * s < d) ? __ldg(r4 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 b = (32 + 4 * s < d) ? __ldg(r4 + 8 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i] = (4 * s + i < d) ? __ldg(row + 4 * s + i) : 0.f;
                v[4 + i] = (32 + 4 * s + i < d) ? __ldg(row + 32 + 4 * s + i) : 0.f;
            }
        }
        if (cosine) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if ((i < 4 ? 4 * s + i : 28 + 4 * s + i) == d) v[i] = 0.f;
        }
    };

    float xv[8];
    load8(R + qr * rs, xv);
    const bool fq = cosine && R[qr * rs + d] != 0.f;

    float key[E];
    int id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = e * 32 + lane;
        int row = -1;   // this lane's candidate: its row in R, -1 for none
        id[e] = INT_MAX;
        if (c < C) {
            const int sp = c / KC, slot = c - sp * KC;
            const int32_t jp = cand[((int64_t)sp * n + q) * KC + slot];
            if (jp >= 0 && (int64_t)jp < n) {   // ids outside [0, n) (an aborted search) are skipped
                const int32_t j = perm ? perm[jp] : jp;   // original id
                row = r_by_pos ? jp : j;
                id[e] = j;
            }
        }
        key[e] = INFINITY;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            // an empty slot scores row 0 and is dropped below (no branch)
            const int yr = max(__shfl_sync(0xffffffffu, row, 4 * g + r), 0);
            float yv[8];
            load8(R + (int64_t)yr * rs, yv);
            float part = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float diff = xv[i] - yv[i];
                part = fmaf(diff, diff, part);
            }
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            part += __shfl_xor_sync(0xffffffffu, part, 4);
            const float got = __shfl_sync(0xffffffffu, part, 8 * (lane & 3));
            if ((lane >> 2) == g && row >= 0) key[e] = got;
        }
        if (cosine && row >= 0) {
            const bool fy = __ldg(R + (int64_t)row * rs + d) != 0.f;
            if (fq || fy) key[e] = (fq && fy) ? 0.f : 2.f;
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
    if (d < 1 || d > 64) return cudaErrorInvalidValue;   // 8 lanes x 8 components per row
    // vector loads when every row starts on a 16-byte boundary
    const bool vec = rs % 4 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0;
#define RSC_RR(e)                                                                                                    \
    case 32 * e:                                                                                                     \
        rerank_kernel<e><<<blocks, kWarps * 32, 0, st>>>(R, rs, n, d, metric, vec, cand, KC, C, k, perm, r_by_pos, \
                                                         idx, dist);                                                 \
        break
    switch (C2) {
        RSC_RR(1); RSC_RR(2); RSC_RR(4); RSC_RR(8); RSC_RR(16); RSC_RR(32);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_RR
    return cudaGetLastError();
}

}  // namespace rsc
