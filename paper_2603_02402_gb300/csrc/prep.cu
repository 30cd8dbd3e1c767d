// Prep pass: one read of X, one write of the padded FP32 operand rows.
//
// Euclidean rows are centred on the column means first: distances do not
// change, but |y|^2 shrinks, and with it the cancellation in the expansion
// form |y|^2 - 2 x.y that the candidate search ranks by.  Cosine distance
// (paper, Methods, "Custom GPU kernels": 1 - x.y/(|x||y|)) is computed on rows
// normalised here, so later steps work with unit vectors:
// 1 - cos = |x^ - y^|^2 / 2.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

constexpr int kRowsPerWarp = 32;
constexpr int kWarps = 4;
constexpr int kColBlocks = 1216;   // 8 per SM: enough loads in flight to stream X near the HBM rate
constexpr int kColTile = 64;   // rows staged in shared memory at a time

// Column sums, deterministic: block b owns a fixed row range (a multiple of 4
// rows long, so every tile of a 16-byte aligned X starts on a 16-byte
// boundary); tiles of kColTile rows are staged in shared memory (16-byte
// loads when X is aligned), and thread (g, c) adds column c of rows g, g + 4,
// ... in order with Kahan compensation.
__global__ void __launch_bounds__(256)
colsum_partials_kernel(const float *__restrict__ X, int64_t n, int d, float *__restrict__ part) {
    __shared__ float red[4][64];
    __shared__ __align__(16) float tile[kColTile * 64];
    const int g = threadIdx.x >> 6, c = threadIdx.x & 63;
    const int64_t chunk = ceil_div(ceil_div(n, gridDim.x), 4) * 4;
    const int64_t r0 = min(n, (int64_t)blockIdx.x * chunk), r1 = min(n, r0 + chunk);
    float s = 0.f, comp = 0.f;
    for (int64_t t0 = r0; t0 < r1; t0 += kColTile) {
        const int rows = (int)min((int64_t)kColTile, r1 - t0);
        const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0;   // caller's rows on 16 bytes
        const int total = rows * d, total4 = vec ? total / 4 : 0;
        const float4 *src4 = reinterpret_cast<const float4 *>(X + t0 * d);
        __syncthreads();
        for (int f = threadIdx.x; f < total4; f += blockDim.x) reinterpret_cast<float4 *>(tile)[f] = src4[f];
        for (int e = 4 * total4 + threadIdx.x; e < total; e += blockDim.x) tile[e] = X[t0 * d + e];
        __syncthreads();
        if (c < d) {
            for (int r = g; r < rows; r += 4) {
                const float y = tile[r * d + c] - comp;
                const float t = s + y;
                comp = (t - s) - y;
                s = t;
            }
        }
    }
    red[g][c] = s - comp;
    __syncthreads();
    if (g == 0 && c < d) part[(int64_t)blockIdx.x * 64 + c] = (red[0][c] + red[1][c]) + (red[2][c] + red[3][c]);
}

// Thread (g, c) adds column c of partials g, g + 4, ... with Kahan
// compensation; the four sums are added in a fixed order.
__global__ void __launch_bounds__(256) colmean_final_kernel(const float *__restrict__ part, int nb, int64_t n,
                                                            int d, float *__restrict__ mu) {
    __shared__ float red[4][64];
    const int g = threadIdx.x >> 6, c = threadIdx.x & 63;
    float s = 0.f, comp = 0.f;
    if (c < d) {
        for (int b = g; b < nb; b += 4) {
            const float y = part[b * 64 + c] - comp;
            const float t = s + y;
            comp = (t - s) - y;
            s = t;
        }
    }
    red[g][c] = s - comp;
    __syncthreads();
    if (g == 0 && c < d) mu[c] = (float)((double)((red[0][c] + red[1][c]) + (red[2][c] + red[3][c])) / (double)n);
}

// A warp stages 32 consecutive rows (contiguous in X) through shared memory so
// that both the read of X and the write of Y are coalesced; lane r then
// handles row r on its own.
__global__ void __launch_bounds__(kWarps * 32)
prep_fp32_kernel(const float *__restrict__ X, int64_t n, int d, int DP, int metric,
                 const float *__restrict__ mu, float *__restrict__ Y, float *__restrict__ ny) {
    extern __shared__ float stage[];   // [kWarps][32][DP + 1]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ld = DP + 1;             // odd stride: lane-per-row access is conflict free
    float *s = stage + (size_t)warp * kRowsPerWarp * ld;
    const int64_t row0 = ((int64_t)blockIdx.x * kWarps + warp) * kRowsPerWarp;
    if (row0 >= n) return;
    const int rows = (n - row0 < kRowsPerWarp) ? (int)(n - row0) : kRowsPerWarp;

    const float *src = X + row0 * d;
    if ((rows * d) % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) {   // 16-byte loads
        const float4 *src4 = reinterpret_cast<const float4 *>(src);
        for (int f = lane; f < rows * d / 4; f += 32) {
            const float4 v = src4[f];
            const int e = 4 * f;
            s[(e / d) * ld + (e % d)] = v.x;
            s[((e + 1) / d) * ld + ((e + 1) % d)] = v.y;
            s[((e + 2) / d) * ld + ((e + 2) % d)] = v.z;
            s[((e + 3) / d) * ld + ((e + 3) % d)] = v.w;
        }
    } else {
        for (int e = lane; e < rows * d; e += 32) s[(e / d) * ld + (e % d)] = src[e];
    }
    __syncwarp();

    if (lane < rows) {
        float *r = s + lane * ld;
        float sum = 0.f;
        for (int t = 0; t < d; ++t) sum = fmaf(r[t], r[t], sum);
        if (metric == RSC_COSINE) {
            if (sum > 0.f) {
                const float nrm = sqrtf(sum);
                for (int t = 0; t < d; ++t) r[t] = r[t] / nrm;
            }
            for (int t = d; t < DP; ++t) r[t] = 0.f;
            r[d] = (sum > 0.f) ? 0.f : 1.f;   // all-zero row flag
            ny[row0 + lane] = 0.f;
        } else {
            float cs = 0.f;
            for (int t = 0; t < d; ++t) {
                r[t] = r[t] - mu[t];
                cs = fmaf(r[t], r[t], cs);
            }
            for (int t = d; t < DP; ++t) r[t] = 0.f;
            ny[row0 + lane] = cs;
        }
    }
    __syncwarp();

    float *dst = Y + row0 * DP;   // DP is a multiple of 8: 16-byte stores
    float4 *dst4 = reinterpret_cast<float4 *>(dst);
    for (int f = lane; f < rows * DP / 4; f += 32) {
        const int e = 4 * f, r = e / DP, t = e % DP;
        dst4[f] = make_float4(s[r * ld + t], s[r * ld + t + 1], s[r * ld + t + 2], s[r * ld + t + 3]);
    }
}

}  // namespace

size_t prep_scratch_floats() { return (size_t)kColBlocks * 64 + 64; }

cudaError_t launch_prep_fp32(const float *X, int64_t n, int d, int DP, int metric,
                             float *Y, float *ny, float *scratch, cudaStream_t st) {
    float *mu = scratch + (size_t)kColBlocks * 64;
    if (metric == RSC_EUCLIDEAN) {
        colsum_partials_kernel<<<kColBlocks, 256, 0, st>>>(X, n, d, scratch);
        colmean_final_kernel<<<1, 256, 0, st>>>(scratch, kColBlocks, n, d, mu);
    }
    const int64_t rows_per_block = (int64_t)kWarps * kRowsPerWarp;
    const int64_t blocks = ceil_div(n, rows_per_block);
    const size_t smem = sizeof(float) * kWarps * kRowsPerWarp * (DP + 1);
    prep_fp32_kernel<<<(unsigned)blocks, kWarps * 32, smem, st>>>(X, n, d, DP, metric, mu, Y, ny);
    return cudaGetLastError();
}

}  // namespace rsc
