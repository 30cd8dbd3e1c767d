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
//               thread owns one query row's part: tcgen05.ld 32 columns at a
//               time, 3-input min tree per 16 values, threshold test against
//               its register top-k, rare appends to a shared-memory buffer.
//               The row's EG per-part lists together form its candidates.
// Every wait is bounded; on timeout the CTA records RSC_ERR_TIMEOUT, drains
// its in-flight copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "topk.cuh"

namespace rsc {

namespace tck {

constexpr int BM = 128;              // query rows per item (TMEM lanes)
constexpr int BN = 256;              // database rows per stage = accumulator columns
constexpr int NBUF = 2;              // accumulators (NBUF x BN = 512 TMEM columns)
constexpr int QBLK = BM * 128;       // bytes of one 128-row x 64-element bf16 query block
constexpr int DBLK = BN * 128;       // bytes of one 256-row x 64-element bf16 database block
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitBudget = 2000000000LL;   // ~1 s of SM clocks

// EG epilogue warpgroups, each owning kCols = BN / EG columns of every tile;
// KCP = top-k list length per (row, part).
template <int KB, int KCP, int EG>
struct Cfg {
    static constexpr int kCols = BN / EG;
    static constexpr int kEpiThreads = EG * 128;
    static constexpr int kThreads = 64 + kEpiThreads;
    static constexpr int kCap = (EG == 4) ? 24 : 32;         // buffer entries per thread
    static constexpr int kQBytes = KB * QBLK;
    static constexpr int kStageBytes = KB * DBLK;
    static constexpr int kBufBytes = kCap * kEpiThreads * 8;
    static constexpr int kBudget = 224 * 1024 - kQBytes - kBufBytes;
    static constexpr int kStages = (kBudget / kStageBytes) > 6 ? 6 : (kBudget / kStageBytes);
    static constexpr int kBarOff = kQBytes + kStages * kStageBytes + kBufBytes;
    static constexpr int kSmem = kBarOff + 256 + 1024;       // barriers + alignment slack
    static_assert(kStages >= 2, "shared memory too small for two stages");
};

__global__ void __launch_bounds__(256)
prep_bf16_kernel(const float *__restrict__ Y, int64_t n, int d, int DP, int metric, int KB,
                 __nv_bfloat16 *__restrict__ Qb, __nv_bfloat16 *__restrict__ Db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *y = Y + i * DP;
    const int W = 64 * KB;
    float nrm = 0.f;
    for (int t = 0; t < d; ++t) {
        const float q = __bfloat162float(__float2bfloat16_rn(y[t]));
        nrm = fmaf(q, q, nrm);
    }
    __nv_bfloat16 ext_q[3], ext_d[3];
    int n_ext;
    if (metric == RSC_EUCLIDEAN) {
        const __nv_bfloat16 h = __float2bfloat16_rn(nrm);
        const float r1 = nrm - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        const __nv_bfloat16 l = __float2bfloat16_rn(r2);
        ext_q[0] = ext_q[1] = ext_q[2] = __float2bfloat16_rn(1.f);
        ext_d[0] = h;
        ext_d[1] = m;
        ext_d[2] = l;
        n_ext = 3;
    } else {
        const float z = y[d];   // all-zero-row flag written by the FP32 prep
        ext_q[0] = __float2bfloat16_rn(z);
        ext_d[0] = __float2bfloat16_rn(-2.f * z);
        n_ext = 1;
    }
    uint4 *qo = reinterpret_cast<uint4 *>(Qb + i * W);
    uint4 *dout = reinterpret_cast<uint4 *>(Db + i * W);
    for (int t8 = 0; t8 < W / 8; ++t8) {
        __align__(16) __nv_bfloat16 qa[8], da[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int t = t8 * 8 + e;
            __nv_bfloat16 qv = __float2bfloat16_rn(0.f), dv = __float2bfloat16_rn(0.f);
            if (t < d) {
                qv = __float2bfloat16_rn(y[t]);
                dv = __float2bfloat16_rn(-2.f * __bfloat162float(qv));   // exact
            } else if (t < d + n_ext) {
                qv = ext_q[t - d];
                dv = ext_d[t - d];
            }
            qa[e] = qv;
            da[e] = dv;
        }
        qo[t8] = *reinterpret_cast<const uint4 *>(qa);
        dout[t8] = *reinterpret_cast<const uint4 *>(da);
    }
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023);
    return reinterpret_cast<uint8_t *>(a);
}

template <int KB, int KCP, int EG>
__global__ void __launch_bounds__(Cfg<KB, KCP, EG>::kThreads, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmD, int64_t n,
              int splits, int64_t split_len, int n_items, int32_t *__restrict__ cand,
              unsigned int *status) {
    using C = Cfg<KB, KCP, EG>;
    constexpr int S = C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint8_t *sQ = smem;
    uint8_t *sD = smem + C::kQBytes;
    float *bkey = reinterpret_cast<float *>(sD + S * C::kStageBytes);
    int *bid = reinterpret_cast<int *>(bkey + C::kCap * C::kEpiThreads);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::kBarOff);
    uint64_t *full = bars;                     // [S]     database stage loaded
    uint64_t *empty = bars + S;                // [S]     database stage consumed
    uint64_t *acc_full = bars + 2 * S;         // [NBUF]  accumulator ready
    uint64_t *acc_empty = acc_full + NBUF;     // [NBUF]  accumulator drained
    uint64_t *q_full = acc_empty + NBUF;
    uint64_t *q_empty = q_full + 1;
    uint64_t *mma_done = q_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(q_full + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NBUF; ++a) {
            tc::mbar_init(&acc_full[a], 1);
            tc::mbar_init(&acc_empty[a], C::kEpiThreads / 32);
        }
        tc::mbar_init(q_full, 1);
        tc::mbar_init(q_empty, 1);
        tc::mbar_init(mma_done, 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        tc::prefetch_tensormap(&tmQ);
        tc::prefetch_tensormap(&tmD);
    }
    if (warp == 1) tc::tmem_alloc<kTmemCols>(tmem_slot);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    // bounded wait: false on timeout (recorded) or when another role aborted
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (tc::mbar_try_wait(bar, parity)) return true;
        const long long t0 = clock64();
        while (true) {
            if (tc::mbar_try_wait(bar, parity)) return true;
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitBudget) {
                *abort_flag = 1;
                record_status(status, RSC_ERR_TIMEOUT);
                return false;
            }
        }
    };
    // bounded wait that ignores the abort flag (draining in-flight work)
    auto drain = [&](uint64_t *bar, uint32_t parity) {
        const long long t0 = clock64();
        while (!tc::mbar_try_wait(bar, parity)) {
            if (clock64() - t0 > kWaitBudget) {
                record_status(status, RSC_ERR_TIMEOUT);
                return;
            }
        }
    };

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            uint32_t gt = 0;
            int item_no = 0;
            bool ok = true, q_issued = false;
            uint32_t q_parity = 0;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++item_no) {
                const int qt = it / splits, sp = it - qt * splits;
                const int64_t j_begin = (int64_t)sp * split_len;
                const int64_t j_end = min(n, j_begin + split_len);
                if (!(ok = wait(q_empty, (item_no & 1) ^ 1))) break;
                tc::mbar_arrive_expect_tx(q_full, C::kQBytes);
                for (int kb = 0; kb < KB; ++kb)
                    tc::tma_load_2d(sQ + kb * QBLK, &tmQ, kb * 64, qt * BM, q_full);
                q_issued = true;
                q_parity = item_no & 1;
                for (int64_t j0 = j_begin; j0 < j_end; j0 += BN, ++gt) {
                    const int s = gt % S;
                    const uint32_t u = gt / S;
                    if (!(ok = wait(&empty[s], (u & 1) ^ 1))) break;
                    tc::mbar_arrive_expect_tx(&full[s], C::kStageBytes);
                    for (int kb = 0; kb < KB; ++kb)
                        tc::tma_load_2d(sD + (s * KB + kb) * DBLK, &tmD, kb * 64, (int)j0, &full[s]);
                }
            }
            if (!ok) {
                // let every copy this thread started land before the CTA exits
                const uint32_t first = gt > (uint32_t)S ? gt - S : 0;
                for (uint32_t t = first; t < gt; ++t) drain(&full[t % S], (t / S) & 1);
                if (q_issued) drain(q_full, q_parity);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
            uint32_t gt = 0;
            int item_no = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++item_no) {
                const int qt = it / splits, sp = it - qt * splits;
                (void)qt;
                const int64_t j_begin = (int64_t)sp * split_len;
                const int64_t j_end = min(n, j_begin + split_len);
                if (!(ok = wait(q_full, item_no & 1))) break;
                tc::tc_fence_after();
                for (int64_t j0 = j_begin; j0 < j_end; j0 += BN, ++gt) {
                    const int s = gt % S;
                    const uint32_t u = gt / S;
                    const uint32_t b = gt % NBUF, v = gt / NBUF;
                    if (!(ok = wait(&acc_empty[b], (v & 1) ^ 1))) break;
                    if (!(ok = wait(&full[s], u & 1))) break;
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + b * BN;
#pragma unroll
                    for (int kb = 0; kb < KB; ++kb) {
                        const uint32_t a_addr = tc::smem_u32(sQ + kb * QBLK);
                        const uint32_t b_addr = tc::smem_u32(sD + (s * KB + kb) * DBLK);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            tc::mma_bf16(d_tmem, tc::smem_desc_sw128(a_addr + kk * 32),
                                         tc::smem_desc_sw128(b_addr + kk * 32), idesc, (kb | kk) != 0);
                        }
                    }
                    tc::mma_commit(&acc_full[b]);   // accumulator ready for the epilogue
                    tc::mma_commit(&empty[s]);      // stage reusable once these MMAs finish
                }
                if (!ok) break;
                tc::mma_commit(q_empty);            // query tile reusable
            }
            tc::mma_commit(mma_done);
            drain(mma_done, 0);
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int e = warp - 2;
        const int part = e >> 2;              // column part of every tile this warp reads
        const int quarter = warp & 3;         // TMEM lane quarter this warp may access
        const int r = quarter * 32 + lane;    // query row within the item
        const uint32_t lane_bits = (uint32_t)(quarter * 32) << 16;
        const int et = threadIdx.x - 64;
        const int cbeg = part * C::kCols;
        BufferedTopK<KCP, C::kCap> tk;
        tk.init(bkey, bid, et, C::kEpiThreads);

        uint32_t gt = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const int qt = it / splits, sp = it - qt * splits;
            const int64_t j_begin = (int64_t)sp * split_len;
            const int64_t j_end = min(n, j_begin + split_len);
            tk.reset();
            for (int64_t j0 = j_begin; j0 < j_end; j0 += BN, ++gt) {
                const uint32_t b = gt % NBUF, v = gt / NBUF;
                ok = wait(&acc_full[b], v & 1);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t tbase = tmem_base + lane_bits + b * BN + cbeg;
                const int valid = ((j_end - j0 < BN) ? (int)(j_end - j0) : BN) - cbeg;
#pragma unroll 1
                for (int c0 = 0; c0 < C::kCols; c0 += 32) {
                    float vv[32];
                    __syncwarp();
                    tc::tmem_ld32(tbase + c0, vv);
                    tc::tmem_wait_ld();
                    if (c0 + 32 == C::kCols) {
                        // last load of this accumulator part: hand it back to the MMA warp
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
                    }
                    if (valid < c0 + 32) {   // ragged end of the range (warp-uniform)
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i >= valid) vv[i] = INFINITY;
                    }
                    float lo[16], hi[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        lo[i] = vv[i];
                        hi[i] = vv[16 + i];
                    }
                    tk.offer16(lo, (int)(j0 + cbeg + c0));
                    tk.offer16(hi, (int)(j0 + cbeg + c0 + 16));
                }
            }
            if (!ok) break;
            tk.flush();
            const int64_t q = (int64_t)qt * BM + r;
            if (q < n) {
                int32_t *out = cand + ((int64_t)(sp * EG + part) * n + q) * KCP;
#pragma unroll
                for (int c = 0; c < KCP; ++c) out[c] = tk.list.id[c];
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tc::tmem_dealloc<kTmemCols>(tmem_base);
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

template <int KB, int KCP, int EG>
cudaError_t launch_kernel(const CUtensorMap &mq, const CUtensorMap &md, int64_t n, int splits, int64_t split_len,
                          int32_t *cand, unsigned int *status, cudaStream_t st) {
    using C = Cfg<KB, KCP, EG>;
    auto kern = knn_tc_kernel<KB, KCP, EG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    const int64_t items = ceil_div(n, BM) * splits;
    const int grid = (int)std::min<int64_t>(items, sm_count());
    kern<<<grid, C::kThreads, C::kSmem, st>>>(mq, md, n, splits, split_len, (int)items, cand, status);
    return cudaGetLastError();
}

}  // namespace tck

int tc_kb(int d, int metric) { return (d + (metric == RSC_EUCLIDEAN ? 3 : 1) <= 64) ? 1 : 2; }

TcShape knn_tc_shape(int d, int metric, int k, int want) {
    // each part's list must be able to hold the whole top-k (all of it may
    // fall in one part), and parts x list >= the requested candidate count
    if (tc_kb(d, metric) == 1 && k <= 16 && want <= 64) return TcShape{4, 16};
    for (int list : {16, 32, 64})
        if (list >= k && 2 * list >= want) return TcShape{2, list};
    return TcShape{0, 0};
}

bool knn_tc_supported(int d, int metric) { return d >= 1 && d + (metric == RSC_EUCLIDEAN ? 3 : 1) <= 128; }

int64_t knn_tc_split_align() { return tck::BN; }

cudaError_t launch_prep_bf16(const float *Y, int64_t n, int d, int DP, int metric, void *Qb, void *Db,
                             cudaStream_t st) {
    const int KB = tc_kb(d, metric);
    tck::prep_bf16_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
        Y, n, d, DP, metric, KB, static_cast<__nv_bfloat16 *>(Qb), static_cast<__nv_bfloat16 *>(Db));
    return cudaGetLastError();
}

cudaError_t launch_knn_tc(const void *Qb, const void *Db, int64_t n, int d, int metric, TcShape sh, int splits,
                          int64_t split_len, int32_t *cand, unsigned int *status, cudaStream_t st) {
    const int KB = tc_kb(d, metric);
    CUtensorMap mq, md;
    cudaError_t e = tck::make_map(&mq, Qb, n, KB, tck::BM);
    if (e != cudaSuccess) return e;
    if ((e = tck::make_map(&md, Db, n, KB, tck::BN)) != cudaSuccess) return e;
#define RSC_TC_CASE(kb, kcp, eg) \
    return tck::launch_kernel<kb, kcp, eg>(mq, md, n, splits, split_len, cand, status, st)
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
