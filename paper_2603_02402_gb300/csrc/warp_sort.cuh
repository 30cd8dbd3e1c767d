// Warp-wide ascending sort of (key, id) pairs held in registers.
//
// E pairs per lane; element v = e * 32 + lane of a virtual array of 32 * E.
// A bitonic network: strides >= 32 compare a lane's own elements, smaller
// strides exchange with lane ^ stride through shuffles.  Order: key, then id
// (the exact-kNN tie rule).  Every lane of the warp must call it.
#pragma once

#include "common.cuh"

namespace rsc {

__device__ __forceinline__ bool pair_gt(float ka, int ia, float kb, int ib) {
    return ka > kb || (ka == kb && ia > ib);
}

template <int E>
__device__ __forceinline__ void warp_sort_pairs(float (&key)[E], int (&id)[E]) {
    const int lane = threadIdx.x & 31;
    constexpr int P = 32 * E;
#pragma unroll
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int es = stride >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ es;
                    if (pe > e) {
                        const bool asc = (((e << 5) | lane) & size) == 0;
                        if (pair_gt(key[e], id[e], key[pe], id[pe]) == asc) {
                            const float tk = key[e];
                            key[e] = key[pe];
                            key[pe] = tk;
                            const int ti = id[e];
                            id[e] = id[pe];
                            id[pe] = ti;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const float pk = __shfl_xor_sync(0xffffffffu, key[e], stride);
                    const int pi = __shfl_xor_sync(0xffffffffu, id[e], stride);
                    const bool asc = (((e << 5) | lane) & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    // the lower position of an ascending pair keeps the smaller pair
                    const bool take =
                        (lower == asc) ? pair_gt(key[e], id[e], pk, pi) : pair_gt(pk, pi, key[e], id[e]);
                    if (take) {
                        key[e] = pk;
                        id[e] = pi;
                    }
                }
            }
        }
    }
}

// Squared distance sum_t (xq_t - y_t)^2 for t < d, accumulated in t order
// (the same rounding whichever loader runs).  w4 > 0: the row is 16-byte
// aligned and its first 4 * w4 floats (w4 <= 16) are read as independent
// float4 loads up front; w4 == 0: scalar loads.
__device__ __forceinline__ float row_dist2(const float *xq, const float *__restrict__ yr, int d, int w4) {
    float acc = 0.f;
    if (w4 > 0) {
        float y[64];
        const float4 *y4 = reinterpret_cast<const float4 *>(yr);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float4 v = (u < w4) ? __ldg(y4 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            y[4 * u] = v.x;
            y[4 * u + 1] = v.y;
            y[4 * u + 2] = v.z;
            y[4 * u + 3] = v.w;
        }
#pragma unroll
        for (int t = 0; t < 64; ++t) {
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

}  // namespace rsc
