#pragma once
// FP32 SIMT candidate search (the plain-precision path).
//
// Brute force over every (query, database row) pair, as exact kNN requires;
// the n x n distances live only in registers.  One thread owns one query row:
// it holds the query in registers, reads database rows from shared memory
// (broadcast), forms s_j = |y_j|^2 - 2 x.y_j (the squared distance minus the
// row constant |x|^2, same order as the distance; paper, Methods, "Custom GPU
// kernels": squared-Euclidean and cosine kernels) and keeps the KC smallest in
// a register top-k.  The exact re-rank in rerank.cu recomputes the final
// distances by direct difference, so the cancellation of the expansion form
// only has to be small next to the gap between candidate k and KC.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "topk.cuh"

namespace rsc {

namespace simt {

constexpr int kThreads = 128;
constexpr int kTileRows = 32;   // database rows per shared-memory tile
constexpr int kChunk = 16;      // values per threshold test
constexpr int kCap = 24;        // candidate buffer entries per thread (>= 16)

template <int DP, int KC>
__global__ void __launch_bounds__(kThreads)
knn_simt_kernel(const float *__restrict__ Y, const float *__restrict__ ny, int64_t n,
                int64_t split_len, int32_t *__restrict__ cand) {
    static_assert(DP % 8 == 0, "DP multiple of 8");
    __shared__ __align__(16) float ys[2][kTileRows][DP];
    __shared__ float ns[2][kTileRows];
    __shared__ float bkey[2 * kCap * kThreads];   // keys, then ids

    const int tid = threadIdx.x;
    const int64_t q = (int64_t)blockIdx.x * kThreads + tid;
    const bool active = q < n;
    const int split = blockIdx.y;
    const int64_t j_begin = (int64_t)split * split_len;
    const int64_t j_end = min(n, j_begin + split_len);

    float x[DP];
    if (active) {
        const float4 *xr = reinterpret_cast<const float4 *>(Y + q * DP);
#pragma unroll
        for (int t4 = 0; t4 < DP / 4; ++t4) {
            const float4 v = xr[t4];
            x[4 * t4 + 0] = v.x;
            x[4 * t4 + 1] = v.y;
            x[4 * t4 + 2] = v.z;
            x[4 * t4 + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int t = 0; t < DP; ++t) x[t] = 0.f;
    }

    BufferedTopK<KC, kCap, kThreads> tk;
    tk.init(bkey, tid);

    // stage tile `buf` with rows j0 .. j0 + kTileRows - 1 (zeros / +inf past the split)
    auto stage = [&](int buf, int64_t j0) {
        constexpr int V4 = kTileRows * DP / 4;
        for (int e = tid; e < V4; e += kThreads) {
            const int r = e / (DP / 4), c4 = e % (DP / 4);
            const int64_t j = j0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < j_end) v = reinterpret_cast<const float4 *>(Y + j * DP)[c4];
            reinterpret_cast<float4 *>(&ys[buf][r][0])[c4] = v;
        }
        if (tid < kTileRows) ns[buf][tid] = (j0 + tid < j_end) ? ny[j0 + tid] : INFINITY;
    };

    int buf = 0;
    if (j_begin < j_end) stage(0, j_begin);
    __syncthreads();
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kTileRows) {
        if (j0 + kTileRows < j_end) stage(buf ^ 1, j0 + kTileRows);   // prefetch next tile
        {   // every lane computes (rows past n on zeros) so the top-k stays warp-synchronous
#pragma unroll
            for (int h = 0; h < kTileRows / kChunk; ++h) {
                float v[kChunk];
#pragma unroll
                for (int i = 0; i < kChunk; ++i) {
                    const float4 *yr = reinterpret_cast<const float4 *>(&ys[buf][h * kChunk + i][0]);
                    float acc = 0.f;
#pragma unroll
                    for (int t4 = 0; t4 < DP / 4; ++t4) {
                        const float4 y4 = yr[t4];
                        acc = fmaf(x[4 * t4 + 0], y4.x, acc);
                        acc = fmaf(x[4 * t4 + 1], y4.y, acc);
                        acc = fmaf(x[4 * t4 + 2], y4.z, acc);
                        acc = fmaf(x[4 * t4 + 3], y4.w, acc);
                    }
                    v[i] = fmaf(-2.f, acc, ns[buf][h * kChunk + i]);
                }
                tk.offer16(v, (int)(j0 + h * kChunk));
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    tk.flush();
    if (active) {
        int32_t *out = cand + ((int64_t)split * n + q) * KC;
#pragma unroll
        for (int c = 0; c < KC; ++c) out[c] = tk.list.id[c];
    }
}

template <int DP, int KC>
cudaError_t launch_t(const float *Y, const float *ny, int64_t n, int splits, int64_t split_len,
                     int32_t *cand, cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(n, kThreads), (unsigned)splits);
    knn_simt_kernel<DP, KC><<<grid, kThreads, 0, st>>>(Y, ny, n, split_len, cand);
    return cudaGetLastError();
}

}  // namespace simt

// One translation unit per KC instantiates every DP (parallel compilation).
template <int KC>
cudaError_t launch_knn_simt_kc(int DP, const float *Y, const float *ny, int64_t n, int splits,
                               int64_t split_len, int32_t *cand, cudaStream_t st);

#define RSC_DEFINE_SIMT_KC(KC)                                                                  \
    template <>                                                                                 \
    cudaError_t launch_knn_simt_kc<KC>(int DP, const float *Y, const float *ny, int64_t n,      \
                                       int splits, int64_t split_len, int32_t *cand,            \
                                       cudaStream_t st) {                                       \
        switch (DP) {                                                                           \
            case 8: return simt::launch_t<8, KC>(Y, ny, n, splits, split_len, cand, st);        \
            case 16: return simt::launch_t<16, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 24: return simt::launch_t<24, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 32: return simt::launch_t<32, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 40: return simt::launch_t<40, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 48: return simt::launch_t<48, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 56: return simt::launch_t<56, KC>(Y, ny, n, splits, split_len, cand, st);      \
            case 64: return simt::launch_t<64, KC>(Y, ny, n, splits, split_len, cand, st);      \
        }                                                                                       \
        return cudaErrorInvalidValue;                                                           \
    }

}  // namespace rsc
