// FP8 (E4M3) tensor-core candidate search: the tcgen05 search of knn_tc.cu
// with 8-bit operands (kind::f8f6f4 MMAs, K = 32 per instruction, 64-byte
// operand rows under a 64-byte swizzle), half the operand bytes and MMA time
// of the BF16 search.  E4M3 keeps 3 mantissa bits, so its candidate lists
// need to be long (see rsc.h); the exact FP32 re-rank restores exact
// distances as for BF16.
//
// Operand rows (64 bytes), with s = 2^e one power-of-two scale for the call
// chosen from the largest |y| so that |s y| <= sqrt(110000 / d):
//   A (queries)  row i: [ q(s y_i), 2^8, 2^4, 2^0, 2^-4, 2^-8, 0 ... ]
//   B (database) row j: [ -2 q(s y_j), b0_j, b1_j, b2_j, b3_j, b4_j, 0 ... ]
// q() = round to E4M3; -2 q() is exact.  The digits b are signed E4M3 values
// with sum_p 2^(8 - 4p) b_p = sum_t q(s y_jt)^2 (each digit takes the rounded
// remainder of the previous ones), so
//   D = A B^T = s^2 ( |y^_j|^2 - 2 y^_i . y^_j ),   y^ = q(s y) / s,
// the squared distance between the rounded points minus a row constant, up to
// the last digit's remainder: the epilogue ranks it as it ranks the BF16
// accumulator.  Cosine rows (unit length): A = [q(s y_i), s z_i], B =
// [-2 q(s y_j), -2 s z_j] with z the all-zero-row flag.
#include <cuda.h>
#include <cuda_fp8.h>
#include <math.h>

#include "knn_tc.cuh"

namespace rsc {

namespace tck {

constexpr int kNormDigits = 5;   // norm digits of weights 2^8, 2^4, 2^0, 2^-4, 2^-8

__device__ __forceinline__ uint8_t to_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float from_e4m3(uint8_t b) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

// Largest |Y[i, t]| over t < d, as the bits of a non-negative float (whose
// order is the integers' order) by atomicMax into *amax (zeroed first).
__global__ void __launch_bounds__(256)
absmax_kernel(const float *__restrict__ Y, int64_t n, int d, int DP, unsigned int *amax) {
    float m = 0.f;
    const int64_t total = n * (int64_t)DP;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        if ((int)(e % DP) < d) m = fmaxf(m, fabsf(Y[e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// Power-of-two scale s = 2^e with s * max|y| <= sqrt(110000 / d): the
// squared norm of a scaled row stays below 110000 < 448 * 256, so its first
// digit (weight 2^8) fits E4M3's largest finite value 448.
__device__ __forceinline__ float fp8_scale(unsigned int amax_bits, int d) {
    const float amax = __uint_as_float(amax_bits);
    if (!(amax > 0.f)) return 1.f;
    const float lim = sqrtf(110000.f / (float)d);
    int e = (int)floorf(log2f(lim / amax));
    e = max(-40, min(40, e));
    return ldexpf(1.f, e);
}

// Thread per row: the 64-byte A and B rows of Y row perm[i] (DP floats).
__global__ void __launch_bounds__(256)
prep_fp8_kernel(const float *__restrict__ Y, int64_t n, int d, int DP, int metric,
                const int32_t *__restrict__ perm, const unsigned int *__restrict__ amax, uint8_t *__restrict__ Qf,
                uint8_t *__restrict__ Df) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = fp8_scale(*amax, d);
    const float *y = Y + (perm ? (int64_t)perm[i] : i) * DP;
    __align__(16) uint8_t qa[64], da[64];
    float nrm = 0.f;
#pragma unroll 8
    for (int t = 0; t < 64; ++t) {
        uint8_t q = 0, dd = 0;
        if (t < d) {
            q = to_e4m3(s * y[t]);
            const float qv = from_e4m3(q);
            dd = to_e4m3(-2.f * qv);   // exact
            nrm = fmaf(qv, qv, nrm);
        }
        qa[t] = q;
        da[t] = dd;
    }
    if (metric == RSC_EUCLIDEAN) {
        float rem = nrm;
#pragma unroll
        for (int p = 0; p < kNormDigits; ++p) {
            const float w = ldexpf(1.f, 8 - 4 * p);
            const uint8_t b = to_e4m3(rem / w);
            rem -= w * from_e4m3(b);
            qa[d + p] = to_e4m3(w);
            da[d + p] = b;
        }
    } else {
        const float z = y[d];   // all-zero-row flag written by the FP32 prep
        qa[d] = to_e4m3(s * z);
        da[d] = to_e4m3(-2.f * s * z);
    }
    uint4 *oq = reinterpret_cast<uint4 *>(Qf + i * 64);
    uint4 *od = reinterpret_cast<uint4 *>(Df + i * 64);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        oq[u] = reinterpret_cast<const uint4 *>(qa)[u];
        od[u] = reinterpret_cast<const uint4 *>(da)[u];
    }
}

}  // namespace tck

bool knn_tc_fp8_supported(int d, int metric) {
    return d >= 1 && d + (metric == RSC_EUCLIDEAN ? tck::kNormDigits : 1) <= 64;
}

cudaError_t launch_prep_fp8(const float *Y, int64_t n, int d, int DP, int metric, const int32_t *perm, void *Qf,
                            void *Df, unsigned int *amax, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    tck::absmax_kernel<<<sm_count() * 8, 256, 0, st>>>(Y, n, d, DP, amax);
    tck::prep_fp8_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(Y, n, d, DP, metric, perm, amax,
                                                                     static_cast<uint8_t *>(Qf),
                                                                     static_cast<uint8_t *>(Df));
    return cudaGetLastError();
}

cudaError_t launch_knn_tc_fp8(const void *Qf, const void *Df, int64_t n, int d, int metric, TcShape sh, int splits,
                              int64_t split_len, int window, int32_t *cand, unsigned int *status, cudaStream_t st) {
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map_fp8(&mq, Qf, n, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map_fp8(&md, Df, n, tck::BN)) != cudaSuccess) return e;
    tck::PlainWork work{n, splits, split_len, cand, (int)(ceil_div(n, tck::BM) * splits), window};
    (void)d;
    (void)metric;
#define RSC_TC_CASE(kcp, eg) return tck::launch_kernel<1, kcp, eg, tck::PlainWork, 1>(mq, md, work, status, st, sh.stages)
    if (sh.parts == 4 && sh.list == 16) RSC_TC_CASE(16, 4);
    if (sh.parts == 2 && sh.list == 16) RSC_TC_CASE(16, 2);
    if (sh.parts == 2 && sh.list == 32) RSC_TC_CASE(32, 2);
    if (sh.parts == 2 && sh.list == 64) RSC_TC_CASE(64, 2);
#undef RSC_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rsc
