#pragma once
// FP32 SIMT candidate search (the plain-precision path).
//
// Brute force over every (query, database row) pair, as exact kNN requires;
// the n x n distances never reach global memory.  For every pair the kernel
// forms s_j = |y_j|^2 - 2 x.y_j (the squared distance minus the row constant
// |x|^2, same order as the distance; paper, Methods, "Custom GPU kernels":
// squared-Euclidean and cosine kernels) by one FMA chain over the components
// in order, and keep the KC smallest per query row in a register top-k.  The
// exact re-rank in rerank.cu recomputes the final distances by direct
// difference, so the cancellation of the expansion form only has to be small
// next to the gap between candidate k and KC.
//
// A register-tiled outer product: 256 queries per CTA against database tiles
// staged transposed in shared memory.  Each thread accumulates an 8 x RB block
// of (query, row) pairs, two 16-byte query loads and RB / 4 row loads per
// component; the block's s values go through a shared 256-query s tile, and
// each thread then scans its own query's row of that tile, in column order, with
// the register top-k.  RB = 8 (64-row tiles) for lists of up to 32; RB = 4
// (32-row tiles) for lists of 64, whose 128 list registers leave no room for
// the 8 x 8 block.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "topk.cuh"

namespace rsc {

namespace simt {

// ----------------------------------------------------- register-tiled kernel

namespace tiled {
constexpr int kThreads = 256;
constexpr int kQ = 256;          // query rows per CTA (one per thread in the scan)
constexpr int kCap = 24;         // candidate buffer entries per thread

// RB database rows per thread: tiles of 8 RB rows; s rows padded by 4 floats
// (16-byte rows, conflict-free scans)
template <int RB>
constexpr int rows() { return 8 * RB; }
template <int RB>
constexpr int pitch() { return 8 * RB + 4; }
template <int DP, int RB>
constexpr size_t smem_bytes() {
    return sizeof(float) * ((size_t)DP * kQ + 2 * DP * rows<RB>() + 2 * rows<RB>() + (size_t)kQ * pitch<RB>() +
                            2 * kCap * kThreads);
}
// 8 rows per thread for lists of up to 32; 4 for lists of 64, whose 128 list
// registers leave room for an 8 x 4 block only
template <int KC>
constexpr int rows_per_thread() { return KC <= 32 ? 8 : 4; }
}  // namespace tiled

// Thread (qg, rg) = (tid / 8, tid % 8) owns queries 4 qg + {0..3} and
// 128 + 4 qg + {0..3} of the CTA and rows 4 rg + {0..3} (and, with RB = 8,
// 32 + 4 rg + {0..3}) of the tile: per component, the 16-byte loads of a warp
// cover 64 contiguous query bytes and 128 contiguous row bytes (one
// shared-memory wavefront each).  Components at `width` and beyond are zero in
// Y and are skipped: an FMA of two zeros leaves s unchanged.
template <int DP, int KC, int RB>
__global__ void __launch_bounds__(tiled::kThreads, 1)
knn_simt_tiled_kernel(const float *__restrict__ Y, const float *__restrict__ ny, int64_t n, int width,
                      int64_t split_len, int32_t *__restrict__ cand) {
    constexpr int kThreads = tiled::kThreads, kQ = tiled::kQ, kR = tiled::rows<RB>(), kPitch = tiled::pitch<RB>();
    constexpr int kCap = tiled::kCap;
    static_assert(RB == 4 || RB == 8, "4 or 8 rows per thread");
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
        float acc[8][RB];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = 0.f;
        const float *yb = ys + buf * DP * kR;
        auto step = [&](int t) {
            const float4 xa = *reinterpret_cast<const float4 *>(xs + t * kQ + 4 * qg);
            const float4 xb = *reinterpret_cast<const float4 *>(xs + t * kQ + 128 + 4 * qg);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            float yv[RB];
#pragma unroll
            for (int h = 0; h < RB / 4; ++h) {
                const float4 y4 = *reinterpret_cast<const float4 *>(yb + t * kR + 32 * h + 4 * rg);
                yv[4 * h + 0] = y4.x;
                yv[4 * h + 1] = y4.y;
                yv[4 * h + 2] = y4.z;
                yv[4 * h + 3] = y4.w;
            }
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
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
#pragma unroll
        for (int h = 0; h < RB / 4; ++h) {
            const float4 nv = *reinterpret_cast<const float4 *>(nys + buf * kR + 32 * h + 4 * rg);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                float *row = S + (a < 4 ? 4 * qg + a : 128 + 4 * qg + a - 4) * kPitch;
                *reinterpret_cast<float4 *>(row + 32 * h + 4 * rg) =
                    make_float4(fmaf(-2.f, acc[a][4 * h + 0], nv.x), fmaf(-2.f, acc[a][4 * h + 1], nv.y),
                                fmaf(-2.f, acc[a][4 * h + 2], nv.z), fmaf(-2.f, acc[a][4 * h + 3], nv.w));
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
    constexpr int RB = tiled::rows_per_thread<KC>();
    constexpr size_t smem = tiled::smem_bytes<DP, RB>();
    auto kern = knn_simt_tiled_kernel<DP, KC, RB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(n, tiled::kQ), (unsigned)splits);
    kern<<<grid, tiled::kThreads, smem, st>>>(Y, ny, n, width, split_len, cand);
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
