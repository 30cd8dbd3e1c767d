// Tensor-core GEMM for the partitioner network (BF16 operands, FP32
// accumulation in tensor memory), sm_103a.
//
//   C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]),
//   A(m, k) = A[m * sam + k * sak],  B(k, n) = B[k * sbk + n * sbn]
//
// Operands come in FP32 with arbitrary strides (the forward pass multiplies
// activations by weights, the backward pass transposed gradients by
// activations), are passed through ReLU where asked and rounded to BF16 while
// the CTA's 128 threads stage them into shared memory in the K-major
// 128-byte-swizzled layout the tensor core reads (one 16-byte chunk of 8 k
// per store; consecutive threads take consecutive rows, so a stride-1 row or
// column dimension is read coalesced either way).  One thread issues
// tcgen05.mma M = 128, N = TN, K = 16 into a TN-column TMEM accumulator; two
// shared-memory stages let the next K block be staged while the tensor core
// consumes the current one.  Every warp reads its 32 TMEM lanes back with
// tcgen05.ld, adds the bias and stores its rows of C.  Every wait is bounded.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsc {
namespace mlp {

constexpr int kTM = 128;                              // C rows per CTA (TMEM lanes)
constexpr int kThreads = 128;
constexpr long long kWaitBudget = 2000000000LL;       // ~1 s of SM clocks
enum { kReluA = 4, kReluB = 8 };                       // same bits as the partitioner's GEMM flags

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Byte offset of 16-byte chunk `ch` (k = 8 ch .. 8 ch + 7) of row r in a
// K-major tile of 128-byte rows under the 128-byte swizzle (8-row groups
// 1024 bytes apart, chunk index XOR row-in-group).
__device__ __forceinline__ uint32_t swz128(int r, int ch) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, unsigned int *status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait_sleep(bar, parity, 2000)) {
        if (clock64() - t0 > kWaitBudget) {
            record_status(status, RSC_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Rows [r0, r0 + R) x k block kc of an operand X(row, k) = X[row * s_row + k * s_k]
// staged as BF16 into a swizzled tile.
template <int R>
__device__ __forceinline__ void stage_tile(uint8_t *tile, const float *__restrict__ X, int64_t s_row, int64_t s_k,
                                           int r0, int rows, int k0, int K, bool relu) {
#pragma unroll 2
    for (int c = threadIdx.x; c < R * 8; c += kThreads) {
        const int r = c % R, ch = c / R;
        const int row = r0 + r, k = k0 + 8 * ch;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float x = 0.f;
            if (row < rows && k + e < K) x = X[(int64_t)row * s_row + (int64_t)(k + e) * s_k];
            v[e] = relu ? fmaxf(x, 0.f) : x;
        }
        *reinterpret_cast<uint4 *>(tile + swz128(r, ch)) =
            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
}

template <int TN>
__global__ void __launch_bounds__(kThreads)
tc_gemm_kernel(int M, int N, int K, const float *__restrict__ A, int64_t sam, int64_t sak,
               const float *__restrict__ B, int64_t sbk, int64_t sbn, float *__restrict__ C, int64_t ldc,
               const float *__restrict__ bias, int flags, unsigned int *status) {
    constexpr int kABytes = kTM * 128, kBBytes = TN * 128, kStage = kABytes + kBBytes;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * kStage);   // [2] stage read, [1] all MMAs done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * TN;
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_init(&bars[2], 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc<TN>(tmem_slot);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, TN);
    const int nk = (K + 63) / 64;
    for (int kc = 0; kc < nk; ++kc) {
        const int b = kc & 1;
        uint8_t *sa = smem + b * kStage;
        // the MMAs that last read this stage (K block kc - 2) must be done
        bool ok = kc < 2 || wait_bar(&bars[b], ((kc - 2) >> 1) & 1, status);
        if (!__syncthreads_and(ok)) break;
        stage_tile<kTM>(sa, A, sam, sak, m0, M, kc * 64, K, (flags & kReluA) != 0);
        stage_tile<TN>(sa + kABytes, B, sbn, sbk, n0, N, kc * 64, K, (flags & kReluB) != 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged bytes visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t a_addr = tc::smem_u32(sa), b_addr = tc::smem_u32(sa + kABytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc_sw128(a_addr + kk * 32), tc::smem_desc_sw128(b_addr + kk * 32),
                             idesc, (kc | kk) != 0);
            tc::mma_commit(&bars[b]);
        }
    }
    // every MMA issued so far has completed once bars[2] completes its phase
    if (tid == 0) tc::mma_commit(&bars[2]);
    const bool done = wait_bar(&bars[2], 0, status);
    tc::tc_fence_after();
    if (__syncthreads_and(done)) {
        const int r = warp * 32 + lane, m = m0 + r;
        const uint32_t lane_bits = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 32) {
            float v[32];
            __syncwarp();
            tc::tmem_ld32(tmem + lane_bits + c0, v);
            tc::tmem_wait_ld();
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int nn = n0 + c0 + j;
                    if (nn < N) C[(int64_t)m * ldc + nn] = v[j] + (bias ? bias[nn] : 0.f);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc<TN>(tmem);
}

template <int TN>
cudaError_t launch(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B,
                   int64_t sbk, int64_t sbn, float *C, int64_t ldc, const float *bias, int flags,
                   unsigned int *status) {
    constexpr int kSmem = 2 * (kTM * 128 + TN * 128) + 64 + 1024;
    auto kern = tc_gemm_kernel<TN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(N, TN), (unsigned)ceil_div(M, kTM));
    kern<<<grid, kThreads, kSmem, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags, status);
    return cudaGetLastError();
}

}  // namespace mlp

cudaError_t launch_tc_gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                           const float *B, int64_t sbk, int64_t sbn, float *C, int64_t ldc, const float *bias,
                           int flags, unsigned int *status) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (N > 128) return mlp::launch<256>(st, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags, status);
    return mlp::launch<128>(st, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, flags, status);
}

}  // namespace rsc
