#pragma once
// FP32 SIMT candidate search (the plain-precision path).
//
// Brute force over every (query, database row) pair, as exact kNN requires;
// the n x n distances never reach global memory.  For every pair the kernels
// form s_j = |y_j|^2 - 2 x.y_j (the squared distance minus the row constant
// |x|^2, same order as the distance; paper, Methods, "Custom GPU kernels":
// squared-Euclidean and cosine kernels) by one FMA chain over the components
// in order, and keep the KC smallest per query row in a register top-k.  The
// exact re-rank in rerank.cu recomputes the final distances by direct
// difference, so the cancellation of the expansion form only has to be small
// next to the gap between candidate k and KC.
//
// Two kernels compute the same s_j, bit for bit, and offer them to the same
// top-k in the same column order, so their lists are identical:
//   knn_simt_tiled_kernel (lists of 16 and 32)  a register-tiled outer product:
//       256 queries per CTA, 64-row database tiles in shared memory; each
//       thread accumulates an 8 x 8 block of (query, row) pairs from two
//       16-byte loads of each side per component (4 loads per 64 FMAs), the
//       block's s values go through a shared 256 x 64 tile, and each thread
//       then scans its own query's row of that tile;
//   knn_simt_kernel (lists of 64, whose 128 list registers leave no room for
//       the 8 x 8 block)  one thread per query, the query in registers, one
//       16-byte broadcast load per 4 FMAs.
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

// ----------------------------------------------------- register-tiled kernel

namespace tiled {
constexpr int kThreads = 256;
constexpr int kQ = 256;          // query rows per CTA (one per thread in the scan)
constexpr int kR = 64;           // database rows per tile
constexpr int kPitch = kR + 4;   // floats per row of the s tile (16-byte rows, conflict-free scans)
constexpr int kCap = 24;         // candidate buffer entries per thread

template <int DP>
constexpr size_t smem_bytes() {
    return sizeof(float) * ((size_t)DP * kQ + 2 * DP * kR + 2 * kR + (size_t)kQ * kPitch + 2 * kCap * kThreads);
}
}  // namespace tiled

// Thread (qg, rg) = (tid / 8, tid % 8) owns queries 4 qg + {0..3} and
// 128 + 4 qg + {0..3} of the CTA and rows 4 rg + {0..3} and 32 + 4 rg + {0..3}
// of the tile: per component, the 16-byte loads of a warp cover 64 contiguous
// query bytes and 128 contiguous row bytes (one shared-memory wavefront each).
// Components at `width` and beyond are zero in Y and are skipped: an FMA of
// two zeros leaves s unchanged.
template <int DP, int KC>
__global__ void __launch_bounds__(tiled::kThreads, 1)
knn_simt_tiled_kernel(const float *__restrict__ Y, const float *__restrict__ ny, int64_t n, int width,
                      int64_t split_len, int32_t *__restrict__ cand) {
    constexpr int kThreads = tiled::kThreads, kQ = tiled::kQ, kR = tiled::kR, kPitch = tiled::kPitch;
    constexpr int kCap = tiled::kCap;
    static_assert(DP % 8 == 0 && DP >= 8, "DP multiple of 8");
    constexpr int C4 = DP / 4;                                   // 16-byte pieces per row
    constexpr int PF = (kR * C4 + kThreads - 1) / kThreads;      // pieces per thread per tile
    extern __shared__ __align__(16) float sm[];
    float *xs = sm;                        // [DP][kQ]    query components, transposed
    float *ys = xs + DP * kQ;              // [2][DP][kR] database tiles, transposed
    float *nys = ys + 2 * DP * kR;         // [2][kR]     |y_j|^2 (+inf past the split)
    float *S = nys + 2 * kR;               // [kQ][kPitch] s values of the current tile
    float *bkey = S + kQ * kPitch;         // top-k buffers

    const int tid = threadIdx.x;
    const int qg = tid >> 3, rg = tid & 7;
    const int64_t q0 = (int64_t)blockIdx.x * kQ;
    const int64_t j_begin = (int64_t)blockIdx.y * split_len;
    const int64_t j_end = min(n, j_begin + split_len);

    for (int e = tid; e < kQ * C4; e += kThreads) {   // lanes take consecutive queries: conflict-free stores
        const int q = e % kQ, c4 = e / kQ;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q0 + q < n) v = reinterpret_cast<const float4 *>(Y + (q0 + q) * DP)[c4];
        xs[(4 * c4 + 0) * kQ + q] = v.x;
        xs[(4 * c4 + 1) * kQ + q] = v.y;
        xs[(4 * c4 + 2) * kQ + q] = v.z;
        xs[(4 * c4 + 3) * kQ + q] = v.w;
    }

    float4 pf[PF];   // the next tile, held in registers while the current one is multiplied
    float pny = INFINITY;
    auto fetch = [&](int64_t j0) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = tid + i * kThreads, r = e % kR, c4 = e / kR;
            pf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c4 < C4 && j0 + r < j_end) pf[i] = reinterpret_cast<const float4 *>(Y + (j0 + r) * DP)[c4];
        }
        if (tid < kR) pny = (j0 + tid < j_end) ? ny[j0 + tid] : INFINITY;
    };
    auto put = [&](int b) {
        float *yb = ys + b * DP * kR;
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = tid + i * kThreads, r = e % kR, c4 = e / kR;
            if (c4 < C4) {
                yb[(4 * c4 + 0) * kR + r] = pf[i].x;
                yb[(4 * c4 + 1) * kR + r] = pf[i].y;
                yb[(4 * c4 + 2) * kR + r] = pf[i].z;
                yb[(4 * c4 + 3) * kR + r] = pf[i].w;
            }
        }
        if (tid < kR) nys[b * kR + tid] = pny;
    };

    BufferedTopK<KC, kCap, kThreads> tk;
    tk.init(bkey, tid);

    int buf = 0;
    if (j_begin < j_end) {
        fetch(j_begin);
        put(0);
    }
    __syncthreads();
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kR) {
        const bool more = j0 + kR < j_end;   // uniform over the CTA
        if (more) fetch(j0 + kR);
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
        const float *yb = ys + buf * DP * kR;
        auto step = [&](int t) {
            const float4 xa = *reinterpret_cast<const float4 *>(xs + t * kQ + 4 * qg);
            const float4 xb = *reinterpret_cast<const float4 *>(xs + t * kQ + 128 + 4 * qg);
            const float4 ya = *reinterpret_cast<const float4 *>(yb + t * kR + 4 * rg);
            const float4 yc = *reinterpret_cast<const float4 *>(yb + t * kR + 32 + 4 * rg);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float yv[8] = {ya.x, ya.y, ya.z, ya.w, yc.x, yc.y, yc.z, yc.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
        };
        // eight components per loop trip: a fully unrolled body outgrows the
        // instruction cache (stalls on instruction fetch dominated)
#pragma unroll 1
        for (int t8 = 0; t8 < DP - 8; t8 += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) step(t8 + u);
        }
#pragma unroll 1
        for (int t = DP - 8; t < width; ++t) step(t);
        __syncthreads();   // every read of ys[buf] and of the previous s tile is done
        {
            const float4 na = *reinterpret_cast<const float4 *>(nys + buf * kR + 4 * rg);
            const float4 nc = *reinterpret_cast<const float4 *>(nys + buf * kR + 32 + 4 * rg);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                float *row = S + (a < 4 ? 4 * qg + a : 128 + 4 * qg + a - 4) * kPitch;
                *reinterpret_cast<float4 *>(row + 4 * rg) =
                    make_float4(fmaf(-2.f, acc[a][0], na.x), fmaf(-2.f, acc[a][1], na.y),
                                fmaf(-2.f, acc[a][2], na.z), fmaf(-2.f, acc[a][3], na.w));
                *reinterpret_cast<float4 *>(row + 32 + 4 * rg) =
                    make_float4(fmaf(-2.f, acc[a][4], nc.x), fmaf(-2.f, acc[a][5], nc.y),
                                fmaf(-2.f, acc[a][6], nc.z), fmaf(-2.f, acc[a][7], nc.w));
            }
        }
        if (more) put(buf ^ 1);
        __syncthreads();   // the s tile and the next database tile are in place
        const float *sr = S + tid * kPitch;
#pragma unroll
        for (int h = 0; h < kR / 16; ++h) {
            float v[16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 w = *reinterpret_cast<const float4 *>(sr + 16 * h + 4 * c);
                v[4 * c + 0] = w.x;
                v[4 * c + 1] = w.y;
                v[4 * c + 2] = w.z;
                v[4 * c + 3] = w.w;
            }
            tk.offer16(v, (int)(j0 + 16 * h));
        }
        buf ^= 1;
    }
    tk.flush();
    if (q0 + tid < n) {
        int32_t *out = cand + ((int64_t)blockIdx.y * n + q0 + tid) * KC;
#pragma unroll
        for (int c = 0; c < KC; ++c) out[c] = tk.list.id[c];
    }
}

template <int DP, int KC>
cudaError_t launch_t(const float *Y, const float *ny, int64_t n, int width, int splits, int64_t split_len,
                     int32_t *cand, cudaStream_t st) {
    if constexpr (KC <= 32) {
        constexpr size_t smem = tiled::smem_bytes<DP>();
        auto kern = knn_simt_tiled_kernel<DP, KC>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)ceil_div(n, tiled::kQ), (unsigned)splits);
        kern<<<grid, tiled::kThreads, smem, st>>>(Y, ny, n, width, split_len, cand);
    } else {
        dim3 grid((unsigned)ceil_div(n, kThreads), (unsigned)splits);
        knn_simt_kernel<DP, KC><<<grid, kThreads, 0, st>>>(Y, ny, n, split_len, cand);
    }
    return cudaGetLastError();
}

}  // namespace simt

// One translation unit per KC instantiates every DP (parallel compilation).
template <int KC>
cudaError_t launch_knn_simt_kc(int DP, const float *Y, const float *ny, int64_t n, int width, int splits,
                               int64_t split_len, int32_t *cand, cudaStream_t st);

#define RSC_DEFINE_SIMT_KC(KC)                                                                  \
    template <>                                                                                 \
    cudaError_t launch_knn_simt_kc<KC>(int DP, const float *Y, const float *ny, int64_t n,      \
                                       int width, int splits, int64_t split_len, int32_t *cand, \
                                       cudaStream_t st) {                                       \
        switch (DP) {                                                                           \
            case 8: return simt::launch_t<8, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 16: return simt::launch_t<16, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 24: return simt::launch_t<24, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 32: return simt::launch_t<32, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 40: return simt::launch_t<40, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 48: return simt::launch_t<48, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 56: return simt::launch_t<56, KC>(Y, ny, n, width, splits, split_len, cand, st); \
            case 64: return simt::launch_t<64, KC>(Y, ny, n, width, splits, split_len, cand, st); \
        }                                                                                       \
        return cudaErrorInvalidValue;                                                           \
    }

}  // namespace rsc
