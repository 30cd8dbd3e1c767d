// Exclusive scan of a count array in two launches (device-wide, any length).
//
// Launch 1: block b adds up segment b of the counts.  Launch 2: block b adds
// up the totals of the segments before it (there are at most kMaxSegs) and
// scans its own segment from there, kTile entries per step with kPer
// consecutive entries per thread.  out[N] = total; with `overflow`
// set, *overflow = total > cap.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace rsc {
namespace seg_scan {

constexpr int kThreads = 1024;
constexpr int kPer = 4;
constexpr int64_t kTile = (int64_t)kThreads * kPer;
constexpr int kMaxSegs = 1024;

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // ws may still be read by an earlier call
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    int64_t t = lane < (kThreads >> 5) ? ws[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

template <class In>
__global__ void __launch_bounds__(kThreads) sum_kernel(const In *__restrict__ cnt, int64_t N, int64_t seg,
                                                       int64_t *__restrict__ sums) {
    __shared__ int64_t ws[32];
    const int64_t b0 = (int64_t)blockIdx.x * seg, b1 = min(N, b0 + seg);
    int64_t s = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kThreads) s += (int64_t)cnt[i];
    s = block_sum(s, ws);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

template <class In, class Out>
__global__ void __launch_bounds__(kThreads) scan_kernel(const In *__restrict__ cnt, int64_t N, int64_t seg,
                                                        const int64_t *__restrict__ sums, Out *__restrict__ out,
                                                        int64_t cap, int32_t *__restrict__ overflow) {
    __shared__ int64_t ws[32];
    __shared__ int64_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t c = 0;
    for (int b = tid; b < (int)blockIdx.x; b += kThreads) c += sums[b];
    c = block_sum(c, ws);
    if (tid == 0) carry_s = c;
    const int64_t b0 = (int64_t)blockIdx.x * seg, b1 = min(N, b0 + seg);
    for (int64_t base = b0; base < b1; base += kTile) {
        const int64_t i0 = base + (int64_t)tid * kPer;
        int64_t v[kPer];
        int64_t x = 0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            v[u] = i0 + u < b1 ? (int64_t)cnt[i0 + u] : 0;
            x += v[u];
        }
        const int64_t own = x;
        for (int o = 1; o < 32; o <<= 1) {   // inclusive warp scan of the threads' sums
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();   // carry_s written, ws free
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < (kThreads >> 5) ? ws[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const int64_t carry = carry_s;
        int64_t run = carry + x - own + (warp > 0 ? ws[warp - 1] : 0);
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            if (i0 + u < b1) out[i0 + u] = (Out)run;
            run += v[u];
        }
        __syncthreads();   // every thread has read carry_s
        if (tid == kThreads - 1) carry_s = run;
    }
    if (blockIdx.x == gridDim.x - 1) {
        __syncthreads();
        if (tid == 0) {
            out[N] = (Out)carry_s;
            if (overflow) *overflow = carry_s > cap ? 1 : 0;
        }
    }
}

// Segment length: whole tiles, at most kMaxSegs segments.
inline int64_t seg_len(int64_t N) {
    const int64_t per = ceil_div(std::max<int64_t>(N, 1), kMaxSegs);
    return std::max<int64_t>(4 * kTile, ceil_div(per, kTile) * kTile);
}

// sums: kMaxSegs int64 of scratch.
template <class In, class Out>
cudaError_t launch(const In *cnt, int64_t N, Out *out, int64_t *sums, cudaStream_t st, int64_t cap = 0,
                   int32_t *overflow = nullptr) {
    const int64_t seg = seg_len(N);
    const unsigned B = (unsigned)std::max<int64_t>(1, ceil_div(N, seg));
    sum_kernel<In><<<B, kThreads, 0, st>>>(cnt, N, seg, sums);
    scan_kernel<In, Out><<<B, kThreads, 0, st>>>(cnt, N, seg, sums, out, cap, overflow);
    return cudaGetLastError();
}

}  // namespace seg_scan
}  // namespace rsc
