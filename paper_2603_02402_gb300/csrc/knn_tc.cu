// BF16 tensor-core candidate search (tcgen05 + TMA + TMEM), sm_103a.
//
// The n x n distance matrix is a dense contraction over the principal
// components (paper, Methods, "Custom GPU kernels": pairwise squared-Euclidean
// and cosine distance kernels), so it runs on the 5th-generation tensor cores
// and never leaves the SM:
//
//   A (queries)  row i: [ bf16(y_i), 1, 1, 1, 0 ... ]              (K = 64)
//   B (database) row j: [ -2 bf16(y_j), h_j, m_j, l_j, 0 ... ]
//   D = A B^T  =  |y^_j|^2 - 2 y^_i . y^_j
//
// with h + m + l a three-piece BF16 split of |y^_j|^2 (FP32, from the rounded
// row), so the accumulator already holds the squared distance between the
// rounded points minus the row constant |y^_i|^2: the epilogue only ranks.
// Cosine rows (unit length) use A = [y^_i, z_i], B = [-2 y^_j, -2 z_j] with z
// the all-zero-row flag.  The exact FP32 re-rank (rerank.cu) restores exact
// distances; this pass only has to bring the true neighbours into the
// per-row candidate list.
//
// One persistent CTA per SM; a work item is 128 query rows (one M = 128
// accumulator) against one database range:
//   warp 0      TMA producer: query tile once per item, then 256-row database
//               tiles through a ring of shared-memory stages
//   warp 1      MMA issuer: per database tile, K/16 tcgen05.mma of
//               M = 128, N = 256 (the largest single-CTA shape: the issuing
//               thread and the per-tile barrier round trips, not the tensor
//               pipe, limit smaller shapes) into one of two 256-column TMEM
//               accumulators (2 x 256 = 512 columns)
//   epilogue    EG warpgroups, each owning 256 / EG columns of every tile; a
//               thread owns one query row's part: tcgen05.ld of 32 columns at
//               a time (64 held in registers in the pruned passes of the
//               two-part shape, 16 for 64-entry lists), 3-input min trees,
//               one warp vote, threshold tests against its register top-k,
//               appends to a shared-memory buffer merged into the lists.
//               The row's EG per-part lists together form its candidates.
// Every wait is bounded; on timeout the CTA records RSC_ERR_TIMEOUT, drains
// its in-flight copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>

#include "knn_tc.cuh"

namespace rsc {

namespace tck {

// BF16 operand rows (row stride W = 64 KB elements): query row = bf16(y),
// database row = -2 bf16(y) (exact), then the folded terms (Euclidean: 1, 1, 1
// against |q|^2 split into three BF16 parts; cosine: the zero-row flag
// against -2 flag), zeros to W.  Row i is source row perm[i].  L = W / 8
// lanes per row, 8 components (one 16-byte store per operand) per lane; the
// row's |q|^2 is summed over its lanes by shuffles.  Y rows are DP floats, DP
// a multiple of 8, so a lane's 8 source floats are two aligned float4 loads.
__global__ void __launch_bounds__(256)
prep_bf16_kernel(const float *__restrict__ Y, int64_t n, int d, int DP, int metric, int KB,
                 const int32_t *__restrict__ perm, __nv_bfloat16 *__restrict__ Qb, __nv_bfloat16 *__restrict__ Db) {
    const int W = 64 * KB, L = W / 8, rpw = 32 / L;
    const int lane = threadIdx.x & 31, l = lane % L;
    const int64_t i = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * rpw + lane / L;
    const bool active = i < n;
    const float *y = Y + (active ? (perm ? (int64_t)perm[i] : i) : 0) * DP;
    const int t0 = 8 * l;
    float v[8];
    if (active && t0 < DP) {
        const float4 a = reinterpret_cast<const float4 *>(y + t0)[0], b = reinterpret_cast<const float4 *>(y + t0)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
    __nv_bfloat16 qv[8];
    float part = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        qv[e] = __float2bfloat16_rn(t0 + e < d ? v[e] : 0.f);
        const float q = __bfloat162float(qv[e]);
        part = fmaf(q, q, part);
    }
    for (int o = L >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const float nrm = part;
    __nv_bfloat16 ext_q[3], ext_d[3];
    int n_ext;
    if (metric == RSC_EUCLIDEAN) {
        const __nv_bfloat16 h = __float2bfloat16_rn(nrm);
        const float r1 = nrm - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
        ext_q[0] = ext_q[1] = ext_q[2] = __float2bfloat16_rn(1.f);
        ext_d[0] = h;
        ext_d[1] = m;
        ext_d[2] = lo;
        n_ext = 3;
    } else {
        const float z = active ? y[d] : 0.f;   // all-zero-row flag written by the FP32 prep
        ext_q[0] = __float2bfloat16_rn(z);
        ext_d[0] = __float2bfloat16_rn(-2.f * z);
        n_ext = 1;
    }
    __align__(16) __nv_bfloat16 qa[8], da[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int t = t0 + e;
        __nv_bfloat16 q = __float2bfloat16_rn(0.f), dd = __float2bfloat16_rn(0.f);
        if (t < d) {
            q = qv[e];
            dd = __float2bfloat16_rn(-2.f * __bfloat162float(q));   // exact
        } else if (t < d + n_ext) {
            q = ext_q[t - d];
            dd = ext_d[t - d];
        }
        qa[e] = q;
        da[e] = dd;
    }
    if (active) {
        reinterpret_cast<uint4 *>(Qb + i * W)[l] = *reinterpret_cast<const uint4 *>(qa);
        reinterpret_cast<uint4 *>(Db + i * W)[l] = *reinterpret_cast<const uint4 *>(da);
    }
}

// --------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// [rows, 64 * KB] bf16, box_rows x 64-element boxes, 128-byte swizzle
cudaError_t make_map(CUtensorMap *m, const void *base, int64_t rows, int KB, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)(64 * KB), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(128 * KB)};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// [rows, 64] FP8 bytes, box_rows x 64-byte boxes, 64-byte swizzle
cudaError_t make_map_fp8(CUtensorMap *m, const void *base, int64_t rows, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {64, (cuuint64_t)rows};
    cuuint64_t strides[1] = {64};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace tck

int tc_kb(int d, int metric) { return (d + (metric == RSC_EUCLIDEAN ? 3 : 1) <= 64) ? 1 : 2; }

TcShape knn_tc_shape(int d, int metric, int k, int want, int parts_req) {
    // each part's list must be able to hold the whole top-k (all of it may
    // fall in one part), and parts x list >= the requested candidate count
    const bool four_ok = tc_kb(d, metric) == 1 && k <= 16 && want <= 64;
    if (parts_req == 4) return four_ok ? TcShape{4, 16} : TcShape{0, 0};
    if (parts_req != 0 && parts_req != 2) return TcShape{0, 0};
    TcShape two{0, 0};
    for (int list : {16, 32, 64}) {
        if (list >= k && 2 * list >= want) {
            two = TcShape{2, list};
            break;
        }
    }
    if (parts_req == 2) return two;
    // automatic: two parts of 16 when they cover the request (half the
    // per-tile epilogue overhead per value and half the re-rank of four
    // parts; 1.14x faster at 1M cells, k = 15), else four parts of 16 (short
    // lists insert faster than two of 32), else two longer lists
    if (two.parts != 0 && two.list == 16) return two;
    if (four_ok) return TcShape{4, 16};
    return two;
}

bool knn_tc_supported(int d, int metric) { return d >= 1 && d + (metric == RSC_EUCLIDEAN ? 3 : 1) <= 128; }

int64_t knn_tc_split_align() { return tck::BN; }
int knn_tc_bm() { return tck::BM; }
int knn_tc_bn() { return tck::BN; }

cudaError_t launch_prep_bf16(const float *Y, int64_t n, int d, int DP, int metric, const int32_t *perm, void *Qb,
                             void *Db, cudaStream_t st) {
    const int KB = tc_kb(d, metric);
    const int rows_per_block = 256 / 32 * (32 / (8 * KB));
    tck::prep_bf16_kernel<<<(unsigned)ceil_div(n, rows_per_block), 256, 0, st>>>(
        Y, n, d, DP, metric, KB, perm, static_cast<__nv_bfloat16 *>(Qb), static_cast<__nv_bfloat16 *>(Db));
    return cudaGetLastError();
}

cudaError_t launch_knn_tc(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh, int splits,
                          int64_t split_len, int window, int32_t *cand, unsigned int *status, cudaStream_t st) {
    const int KB = tc_kb(d, metric);
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, n, KB, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, n, KB, tck::BN)) != cudaSuccess) return e;
    tck::PlainWork work{n, splits, split_len, cand, (int)(ceil_div(n, tck::BM) * splits), window};
#define RSC_TC_CASE(kb, kcp, eg) return tck::launch_kernel<kb, kcp, eg>(mq, md, work, status, st, sh.stages)
    if (KB == 1 && sh.parts == 4 && sh.list == 16) RSC_TC_CASE(1, 16, 4);
    if (KB == 1 && sh.parts == 2 && sh.list == 16) RSC_TC_CASE(1, 16, 2);
    if (KB == 1 && sh.parts == 2 && sh.list == 32) RSC_TC_CASE(1, 32, 2);
    if (KB == 1 && sh.parts == 2 && sh.list == 64) RSC_TC_CASE(1, 64, 2);
    if (KB == 2 && sh.parts == 2 && sh.list == 16) RSC_TC_CASE(2, 16, 2);
    if (KB == 2 && sh.parts == 2 && sh.list == 32) RSC_TC_CASE(2, 32, 2);
    if (KB == 2 && sh.parts == 2 && sh.list == 64) RSC_TC_CASE(2, 64, 2);
#undef RSC_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rsc
