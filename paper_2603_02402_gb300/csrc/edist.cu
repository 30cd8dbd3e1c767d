// E-distance group-pair sums on the tensor cores (paper, Methods,
// "Perturbation distance computation"): for every requested group pair
// (a, b), S_ab = sum of ||x_i - x_j|| over i in a, j in b (a != b) or over the
// pairs i < j inside a (a == b, the upper triangle).  Groups are CSR-style
// (offsets into a cell index array); the cells are gathered into group order,
// so the upper triangle of the n x n distance matrix in that order holds every
// pair a <= b, each value belonging to (group of row, group of column).
//
// Distances come from tcgen05 MMAs of BF16 operands with the products split
// into high and low parts, y ~ h + l (h = bf16(y), l = bf16(y - h)), three
// 64-wide K blocks:
//   A row i: [ h_i, 1, 1, 1, n_i^h, n_i^m, n_i^l | l_i | h_i ]
//   B row j: [ -2 h_j, n_j^h, n_j^m, n_j^l, 1, 1, 1 | -2 h_j | -2 l_j ]
// (n^h + n^m + n^l = |y|^2 in three BF16 digits), so the FP32 accumulator is
// |y_i|^2 + |y_j|^2 - 2 (h_i.h_j + l_i.h_j + h_i.l_j) = |y_i - y_j|^2 up to the
// dropped l_i.l_j term (about 2^-18 |y_i| |y_j|) and the FP32 rounding of the
// accumulation.  y = x - c with c the mean of a sample of the rows (distances
// do not depend on c; a small |y| keeps those errors small).  d + 6 <= 64.
//
// Kernel: persistent, warp-specialised like the kNN search.  A TMA warp loads
// the 128-row query tile (three K blocks) once per item and 128-row database
// tiles through a ring of stages; one thread issues the 3 x 4 MMAs of
// M = 128, N = 128, K = 16 per tile into one of two TMEM accumulators;
// sixteen epilogue warps (four TMEM lane quarters x four 32-column chunks)
// take sqrt(|v|) of every value and add it to the current (row group,
// column group) sum.  A chunk table (the group of a chunk's first column and
// the length of its run, loaded one tile ahead) gives the columns' groups; a
// chunk of one group away from the diagonal is summed without predicates.
// A chunk's columns split into runs of one group each (warp-uniform); per run
// a thread adds its FP32 partial to a float-float sum (TwoSum: FP32 pipes
// only), and when the column group changes the warp reduces the sums of rows
// of one group (rows are in group order, so equal groups are adjacent lanes)
// and one lane per run adds them to S with one double atomic.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "knn_tc.cuh"
#include "tc_ptx.cuh"

namespace rsc {

namespace ed {

constexpr int BM = 128;          // query rows per tile (TMEM lanes)
constexpr int BN = 128;          // database rows per tile (accumulator columns)
constexpr int KB = 3;            // 64-wide K blocks: h, l, h against h, h, l
constexpr int kEpiWarps = 16;    // 4 lane quarters x 4 column quarters
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kCols = BN / 4;    // columns per epilogue warp (one 32-column chunk)
constexpr int kQBlk = BM * 128;  // bytes of one 64-element bf16 block of the query tile
constexpr int kDBlk = BN * 128;
constexpr int kQBytes = KB * kQBlk;
constexpr int kStageBytes = KB * kDBlk;
constexpr int kStages = 3;
constexpr int kBarOff = kQBytes + kStages * kStageBytes;
constexpr int kSmem = kBarOff + 256 + 1024;
constexpr uint32_t kTmemCols = 256;   // two accumulators of BN columns
constexpr int kSample = 4096;         // rows averaged for the centre c

// c = mean of up to kSample rows spread over the gathered order (one block;
// thread t sums column t % d over its share of the rows, then the block
// reduces in shared memory).
__global__ void __launch_bounds__(256) centre_kernel(const float *__restrict__ X, const int32_t *__restrict__ cell,
                                                     int64_t n, int64_t n_rows, int d, float *__restrict__ centre) {
    __shared__ float part[256];
    const int m = (int)std::min<int64_t>(n, kSample);
    const int t = threadIdx.x;
    for (int c0 = 0; c0 < d; c0 += 8) {   // 8 columns at a time, 32 threads per column
        const int col = c0 + (t & 7), sl = t >> 3;
        float s = 0.f;
        if (col < d)
            for (int r = sl; r < m; r += 32) {
                const int64_t p = (int64_t)r * n / m;
                int64_t row = cell ? cell[p] : p;
                if (row < 0 || row >= n_rows) row = 0;   // recorded by the prep kernel
                s += X[row * d + col];
            }
        part[t] = s;
        __syncthreads();
        if (t < 8 && c0 + t < d) {
            float a = 0.f;
            for (int k = 0; k < 32; ++k) a += part[k * 8 + t];
            centre[c0 + t] = a / (float)m;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c) {
    a = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// Thread per gathered position p: the A and B operand rows (3 x 128 bytes
// each) of cell cell[p] (or p), and its group.
__global__ void __launch_bounds__(256) prep_kernel(const float *__restrict__ X, const int32_t *__restrict__ cell,
                                                   int64_t n, int64_t n_rows, int d, unsigned int *status,
                                                   const float *__restrict__ centre,
                                                   const int64_t *__restrict__ offsets, int G,
                                                   __nv_bfloat16 *__restrict__ A, __nv_bfloat16 *__restrict__ B,
                                                   int32_t *__restrict__ group) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t row = cell ? cell[p] : p;
    if (row < 0 || row >= n_rows) {   // bad cell index: recorded, row 0 read instead
        record_status(status, RSC_ERR_INVALID_ARG);
        row = 0;
    }
    const float *x = X + row * d;
    __nv_bfloat16 *a = A + p * (64 * KB), *b = B + p * (64 * KB);
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
    float nrm = 0.f;
    for (int t = 0; t < 64; ++t) {
        if (t < d) {
            const float y = x[t] - centre[t];
            nrm = fmaf(y, y, nrm);
            const __nv_bfloat16 h = __float2bfloat16_rn(y);
            const __nv_bfloat16 l = __float2bfloat16_rn(y - __bfloat162float(h));
            const __nv_bfloat16 h2 = __float2bfloat16_rn(-2.f * __bfloat162float(h));   // exact
            const __nv_bfloat16 l2 = __float2bfloat16_rn(-2.f * __bfloat162float(l));   // exact
            a[t] = h;
            a[64 + t] = l;
            a[128 + t] = h;
            b[t] = h2;
            b[64 + t] = h2;
            b[128 + t] = l2;
        } else {
            a[t] = a[64 + t] = a[128 + t] = z;
            b[t] = b[64 + t] = b[128 + t] = z;
        }
    }
    __nv_bfloat16 nh, nm, nl;
    split3(nrm, nh, nm, nl);
    a[d] = a[d + 1] = a[d + 2] = one;
    a[d + 3] = nh;
    a[d + 4] = nm;
    a[d + 5] = nl;
    b[d] = nh;
    b[d + 1] = nm;
    b[d + 2] = nl;
    b[d + 3] = b[d + 4] = b[d + 5] = one;
    int lo = 0, hi = G - 1;   // group of position p: last g with offsets[g] <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    group[p] = lo;
}

// Per 32-column chunk of the gathered order: the group of its first column and
// the length of that group's run inside the chunk (32 when the chunk holds one
// group), so an epilogue warp knows its columns' group with one load.
__global__ void __launch_bounds__(256) chunk_kernel(const int32_t *__restrict__ group,
                                                    const int64_t *__restrict__ offsets, int64_t n,
                                                    int2 *__restrict__ chunk) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c0 = c * 32;
    if (c0 >= n) return;
    const int g = group[c0];
    const int64_t end = std::min(std::min(offsets[g + 1], n), c0 + 32);
    chunk[c] = make_int2(g, (int)(end - c0));
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// hi + lo += x as a float-float pair: Knuth's TwoSum puts the rounding error
// of hi + x into lo, so the pair carries about 48 significant bits (FP32
// pipes only; the FP64 pipe is narrow on this part).
__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// x as a double, built from its bits with integer operations (the FP64 pipe
// is narrow on this part): exact for normal x; zero and subnormal x give 0
// (below 2^-126, far under the sums' resolution); x is finite.
__device__ __forceinline__ double float_bits_to_double(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// Adds the float-float sums of a warp's rows to S[g_row * G + gc]: rows are in
// group order, so lanes of one group are adjacent; a segmented inclusive scan
// over the lanes, then the last lane of each run adds the run's two parts
// to S with FP64 atomics.
__device__ __forceinline__ void flush_sums(float hi, float lo, int grow, int gc, int lane, int G,
                                           double *__restrict__ S) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float vh = __shfl_up_sync(0xffffffffu, hi, o);
        const float vl = __shfl_up_sync(0xffffffffu, lo, o);
        const int g = __shfl_up_sync(0xffffffffu, grow, o);
        if (lane >= o && g == grow) {
            ff_add(hi, lo, vh);
            lo = __fadd_rn(lo, vl);
        }
    }
    const int gn = __shfl_down_sync(0xffffffffu, grow, 1);
    if (grow >= 0 && (lane == 31 || gn != grow)) {
        // the pair's two parts added to S separately (no FP64 arithmetic)
        double *dst = &S[(int64_t)grow * G + gc];
        if (hi != 0.f) atomicAdd(dst, float_bits_to_double(hi));
        if (lo != 0.f) atomicAdd(dst, float_bits_to_double(lo));
    }
}

// Work item: query tile qt against database tiles [dt0, dt1).
struct EdItem {
    int32_t qt, dt0, dt1, pad;
};

__global__ void __launch_bounds__(kThreads, 1)
edist_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const EdItem *__restrict__ items, int n_items, int64_t n, const int32_t *__restrict__ group,
                const int64_t *__restrict__ offsets, const int2 *__restrict__ chunk, int G,
                const uint32_t *__restrict__ pair_bits, double *S, unsigned int *status, long long wait_budget) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = tck::align1024(smem_raw);
    uint8_t *sQ = smem;
    uint8_t *sD = smem + kQBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBarOff);
    uint64_t *full = bars;                     // [kStages]
    uint64_t *empty = bars + kStages;          // [kStages]
    uint64_t *acc_full = bars + 2 * kStages;   // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2]
    uint64_t *q_full = acc_empty + 2;
    uint64_t *q_empty = q_full + 1;
    uint64_t *mma_done = q_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&acc_full[a], 1);
            tc::mbar_init(&acc_empty[a], kEpiWarps);
        }
        tc::mbar_init(q_full, 1);
        tc::mbar_init(q_empty, 1);
        tc::mbar_init(mma_done, 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        tc::prefetch_tensormap(&tmA);
        tc::prefetch_tensormap(&tmB);
    }
    if (warp == 1) tc::tmem_alloc<kTmemCols>(tmem_slot);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const uint32_t sleep_ns = (uint32_t)min((long long)tck::kSleepNs, wait_budget / 4);
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (tc::mbar_try_wait(bar, parity)) return true;
        const long long t0 = clock64();
        while (true) {
            if (tc::mbar_try_wait_sleep(bar, parity, sleep_ns)) return true;
            if (*abort_flag) return false;
            if (clock64() - t0 > wait_budget) {
                *abort_flag = 1;
                record_status(status, RSC_ERR_TIMEOUT);
                return false;
            }
        }
    };
    auto drain = [&](uint64_t *bar, uint32_t parity) {
        const long long t0 = clock64();
        while (!tc::mbar_try_wait(bar, parity)) {
            if (clock64() - t0 > tck::kWaitBudget) {
                record_status(status, RSC_ERR_TIMEOUT);
                return;
            }
        }
    };

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            uint32_t gt = 0;
            tck::StageRing ring;
            ring.S = kStages;
            bool ok = true, q_issued = false;
            uint32_t q_parity = 0;
            int k = 0;
            for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++k) {
                const EdItem wi = items[it];
                if (!(ok = wait(q_empty, (k & 1) ^ 1))) break;
                tc::mbar_arrive_expect_tx(q_full, kQBytes);
                for (int kb = 0; kb < KB; ++kb) tc::tma_load_2d(sQ + kb * kQBlk, &tmA, kb * 64, wi.qt * BM, q_full);
                q_issued = true;
                q_parity = k & 1;
                for (int dt = wi.dt0; dt < wi.dt1; ++dt, ++gt, ring.next()) {
                    const int s = ring.s;
                    if (!(ok = wait(&empty[s], ring.ph ^ 1u))) break;
                    tc::mbar_arrive_expect_tx(&full[s], kStageBytes);
                    for (int kb = 0; kb < KB; ++kb)
                        tc::tma_load_2d(sD + (s * KB + kb) * kDBlk, &tmB, kb * 64, dt * BN, &full[s]);
                }
                if (!ok) break;
            }
            if (!ok) {   // let every copy this thread started land before the CTA exits
                const uint32_t first = gt > (uint32_t)kStages ? gt - kStages : 0;
                for (uint32_t t = first; t < gt; ++t) drain(&full[t % kStages], (t / kStages) & 1);
                if (q_issued) drain(q_full, q_parity);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
            uint32_t gt = 0;
            tck::StageRing ring;
            ring.S = kStages;
            bool ok = true;
            int k = 0;
            for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++k) {
                const EdItem wi = items[it];
                if (!(ok = wait(q_full, k & 1))) break;
                tc::tc_fence_after();
                for (int dt = wi.dt0; dt < wi.dt1; ++dt, ++gt, ring.next()) {
                    const int s = ring.s;
                    const uint32_t b = gt & 1u, v = gt >> 1;
                    if (!(ok = wait(&acc_empty[b], (v & 1) ^ 1))) break;
                    if (!(ok = wait(&full[s], ring.ph))) break;
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + b * BN;
#pragma unroll
                    for (int kb = 0; kb < KB; ++kb) {
                        const uint32_t a_addr = tc::smem_u32(sQ + kb * kQBlk);
                        const uint32_t b_addr = tc::smem_u32(sD + (s * KB + kb) * kDBlk);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc::mma_bf16(d_tmem, tc::smem_desc_sw128(a_addr + kk * 32),
                                         tc::smem_desc_sw128(b_addr + kk * 32), idesc, (kb | kk) != 0);
                    }
                    tc::mma_commit(&acc_full[b]);
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(q_empty);
            }
            tc::mma_commit(mma_done);
            drain(mma_done, 0);
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int e = warp - 2;
        const int part = e >> 2;                 // 32-column chunk of every tile
        const int quarter = warp & 3;            // TMEM lane quarter this warp may access
        const int r = quarter * 32 + lane;       // query row within the tile
        const uint32_t lane_bits = (uint32_t)(quarter * 32) << 16;
        uint32_t gt = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const EdItem wi = items[it];
            const int64_t q0 = (int64_t)wi.qt * BM;
            const int64_t i = q0 + r;                    // gathered position of this thread's row
            const int grow = i < n ? group[i] : -1;
            int gc = -1;          // column group of the open sum (warp-uniform)
            float acc = 0.f, acc_lo = 0.f;   // this row's sum for (grow, gc), float-float
            auto open = [&](int g) {   // make g the open column group (warp-uniform)
                if (g != gc) {
                    if (gc >= 0) flush_sums(acc, acc_lo, grow, gc, lane, G, S);
                    gc = g;
                    acc = 0.f;
                    acc_lo = 0.f;
                }
            };
            auto wanted = [&](int g) -> bool {
                bool w = grow >= 0 && grow <= g;
                if (w && pair_bits) {
                    const int64_t bit = (int64_t)grow * G + g;
                    w = (pair_bits[bit >> 5] >> (bit & 31)) & 1u;
                }
                return w;
            };
            int64_t cbase = (int64_t)wi.dt0 * BN + part * kCols;
            int2 ch = cbase < n ? chunk[cbase >> 5] : make_int2(0, 0);
            for (int dt = wi.dt0; dt < wi.dt1; ++dt, ++gt) {
                const uint32_t b = gt & 1u;
                ok = __all_sync(0xffffffffu, wait(&acc_full[b], (gt >> 1) & 1u));
                if (!ok) break;
                tc::tc_fence_after();
                float v[32];
                __syncwarp();
                tc::tmem_ld32(tmem_base + lane_bits + b * BN + part * kCols, v);
                tc::tmem_wait_ld();
                // the values are in registers: hand the accumulator back to the MMA warp
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
                const int2 cur = ch;
                const int64_t cb = cbase;
                cbase += BN;
                if (dt + 1 < wi.dt1 && cbase < n) ch = chunk[cbase >> 5];   // next tile's chunk, loaded early
#pragma unroll
                // sqrt(|v|): v below 0 is rounding noise of a near-zero squared
                // distance, |v| <= its error bound, so sqrt(|v|) stays within the
                // distance error sqrt(bound) that sqrt(max(0, v)) has, without
                // the comparison
                for (int u = 0; u < 32; ++u) v[u] = sqrt_fast(fabsf(v[u]));
                if (cb >= n) continue;
                const bool diag = cb < q0 + BM;          // some column may not lie above some row
                // columns u with cb + u > i count: u > above, above clamped to
                // [-1, 32] so that the tests are 32-bit
                const int above = (int)max((int64_t)-1, min((int64_t)32, i - cb));
                if (cur.y == 32) {                       // one group over the whole chunk
                    open(cur.x);
                    if (wanted(cur.x)) {
                        float sum = 0.f;
                        if (!diag) {
#pragma unroll
                            for (int u = 0; u < 32; ++u) sum += v[u];
                        } else {
#pragma unroll
                            for (int u = 0; u < 32; ++u) sum += (u > above) ? v[u] : 0.f;
                        }
                        ff_add(acc, acc_lo, sum);
                    }
                    continue;
                }
                const int64_t cend = min(n, cb + kCols);
                for (int64_t c = cb; c < cend;) {        // runs of one column group (warp-uniform)
                    const int g = c == cb ? cur.x : group[c];
                    const int64_t seg_end = c == cb ? cb + cur.y : min(cend, offsets[g + 1]);
                    open(g);
                    if (wanted(g)) {
                        // columns [lo, u1): one unsigned range test per column
                        const int u1 = (int)(seg_end - cb), lo = max((int)(c - cb), above + 1);
                        const unsigned span = u1 > lo ? (unsigned)(u1 - lo) : 0u;
                        float sum = 0.f;
#pragma unroll
                        for (int u = 0; u < 32; ++u) sum += ((unsigned)(u - lo) < span) ? v[u] : 0.f;
                        ff_add(acc, acc_lo, sum);
                    }
                    c = seg_end;
                }
            }
            if (ok && gc >= 0) flush_sums(acc, acc_lo, grow, gc, lane, G, S);
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


// Mean distances and energy distances of the requested pairs (thread per
// (a, b) of the G x G output): mean = S / (n_a n_b), or S / (n_a (n_a - 1) / 2)
// on the diagonal (0 below two cells); E = 2 mean_ab - mean_aa - mean_bb when
// the pair and both diagonals were requested; NaN where not requested.
__global__ void __launch_bounds__(256) assemble_kernel(const double *__restrict__ S, const int64_t *__restrict__ offsets,
                                                       int G, const uint32_t *__restrict__ pair_bits,
                                                       double *__restrict__ mean, double *__restrict__ E) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)G * G) return;
    const int a = (int)(t / G), b = (int)(t - (int64_t)a * G);
    auto requested = [&](int x, int y) -> bool {
        const int lo = min(x, y), hi = max(x, y);
        if (!pair_bits) return true;
        const int64_t bit = (int64_t)lo * G + hi;
        return (pair_bits[bit >> 5] >> (bit & 31)) & 1u;
    };
    auto mean_of = [&](int x, int y) -> double {
        const int lo = min(x, y), hi = max(x, y);
        const double nx = (double)(offsets[lo + 1] - offsets[lo]), ny = (double)(offsets[hi + 1] - offsets[hi]);
        const double s = S[(int64_t)lo * G + hi];
        if (lo == hi) return nx >= 2.0 ? s / (nx * (nx - 1.0) * 0.5) : 0.0;
        return (nx > 0.0 && ny > 0.0) ? s / (nx * ny) : 0.0;
    };
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const bool rq = requested(a, b);
    if (mean) mean[t] = rq ? mean_of(a, b) : nan;
    if (E) E[t] = (rq && requested(a, a) && requested(b, b)) ? 2.0 * mean_of(a, b) - mean_of(a, a) - mean_of(b, b)
                                                            : nan;
}

}  // namespace ed

// ------------------------------------------------------------------- host side

namespace {

constexpr int kChunk = 32;   // database tiles per work item

struct EdPlan {
    int64_t n = 0;                      // gathered cells (offsets[G])
    int G = 0;
    std::vector<ed::EdItem> items;
    std::vector<uint32_t> bits;         // requested pairs (a <= b), empty for all pairs
};

int group_of(const int64_t *off, int G, int64_t p) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

rsc_status plan_edistance(int64_t n_rows, int32_t d, const int64_t *off, int32_t G, const int32_t *pairs,
                          int64_t n_pairs, EdPlan *p) {
    if (n_rows < 1 || n_rows >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "n_rows=%lld", (long long)n_rows);
    if (d < 1 || d > 58) return fail(d > 58 ? RSC_ERR_UNSUPPORTED : RSC_ERR_INVALID_ARG, "d=%d out of [1, 58]", d);
    if (!off || G < 1 || G > 65535) return fail(RSC_ERR_INVALID_ARG, "offsets NULL or n_groups=%d out of [1, 65535]", G);
    if (off[0] != 0) return fail(RSC_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int g = 0; g < G; ++g)
        if (off[g + 1] < off[g]) return fail(RSC_ERR_INVALID_ARG, "offsets decrease at group %d", g);
    if (off[G] < 1 || off[G] >= (int64_t(1) << 31)) return fail(RSC_ERR_INVALID_ARG, "offsets[G]=%lld", (long long)off[G]);
    if (pairs && (n_pairs < 0 || G > 16384))
        return fail(RSC_ERR_INVALID_ARG, "explicit pairs need 0 <= n_pairs and n_groups <= 16384");
    p->n = off[G];
    p->G = G;
    const int64_t n = p->n, T = ceil_div(n, ed::BN);
    std::vector<std::vector<int>> adj;
    if (pairs) {
        p->bits.assign((size_t)ceil_div((int64_t)G * G, 32), 0u);
        adj.resize(G);
        for (int64_t q = 0; q < n_pairs; ++q) {
            const int a = pairs[2 * q], b = pairs[2 * q + 1];
            if (a < 0 || b >= G || a > b) return fail(RSC_ERR_INVALID_ARG, "pair %lld = (%d, %d)", (long long)q, a, b);
            const int64_t bit = (int64_t)a * G + b;
            if (!((p->bits[(size_t)(bit >> 5)] >> (bit & 31)) & 1u)) adj[a].push_back(b);
            p->bits[(size_t)(bit >> 5)] |= 1u << (bit & 31);
        }
        for (auto &v : adj) std::sort(v.begin(), v.end());
    }
    auto emit = [&](int qt, int64_t t0, int64_t t1) {   // tiles [t0, t1) of query tile qt, in chunks
        for (int64_t t = std::max<int64_t>(t0, qt); t < t1; t += kChunk)
            p->items.push_back(ed::EdItem{qt, (int32_t)t, (int32_t)std::min<int64_t>(t1, t + kChunk), 0});
    };
    for (int64_t qt = 0; qt < T; ++qt) {
        if (!pairs) {
            emit((int)qt, qt, T);
            continue;
        }
        const int ga = group_of(off, G, qt * ed::BM), gb = group_of(off, G, std::min(n, (qt + 1) * ed::BM) - 1);
        std::vector<std::pair<int64_t, int64_t>> iv;   // tile intervals of the needed column groups
        for (int a = ga; a <= gb; ++a)
            for (int b : adj[a])
                if (off[b + 1] > off[b]) iv.push_back({off[b] / ed::BN, ceil_div(off[b + 1], ed::BN)});
        std::sort(iv.begin(), iv.end());
        int64_t s0 = -1, s1 = -1;
        for (auto &x : iv) {
            if (x.first > s1) {
                if (s1 > s0) emit((int)qt, s0, s1);
                s0 = x.first;
                s1 = x.second;
            } else {
                s1 = std::max(s1, x.second);
            }
        }
        if (s1 > s0) emit((int)qt, s0, s1);
    }
    // largest items first is unnecessary: chunks are equal but for the last of each band
    return RSC_OK;
}

struct EdLayout {
    unsigned int *status;
    float *centre;
    __nv_bfloat16 *A, *B;
    int32_t *group;
    int2 *chunk;
    int64_t *offsets;
    ed::EdItem *items;
    uint32_t *bits;
};

EdLayout carve_edistance(void *ws, const EdPlan &p, size_t *bytes) {
    Carve cv(ws);
    EdLayout L;
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.centre = cv.take<float>(64);
    L.A = cv.take<__nv_bfloat16>((size_t)p.n * 64 * ed::KB);
    L.B = cv.take<__nv_bfloat16>((size_t)p.n * 64 * ed::KB);
    L.group = cv.take<int32_t>((size_t)p.n);
    L.chunk = cv.take<int2>((size_t)ceil_div(p.n, 32));
    L.offsets = cv.take<int64_t>((size_t)p.G + 1);
    L.items = cv.take<ed::EdItem>(std::max<size_t>(p.items.size(), 1));
    L.bits = p.bits.empty() ? nullptr : cv.take<uint32_t>(p.bits.size());
    if (bytes) *bytes = cv.used;
    return L;
}

// Group sums S[G, G] of the plan (zeroed here).
rsc_status run_edistance_sums(const float *X, int64_t n_rows, int32_t d, const int32_t *cell, const int64_t *off,
                              const EdPlan &p, const EdLayout &L, double *S, cudaStream_t st) {
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, kStatusBytes, st));
    RSC_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(double) * (size_t)p.G * p.G, st));
    RSC_CUDA_TRY(cudaMemcpyAsync(L.offsets, off, sizeof(int64_t) * (p.G + 1), cudaMemcpyHostToDevice, st));
    if (!p.items.empty())
        RSC_CUDA_TRY(cudaMemcpyAsync(L.items, p.items.data(), sizeof(ed::EdItem) * p.items.size(),
                                     cudaMemcpyHostToDevice, st));
    if (L.bits)
        RSC_CUDA_TRY(cudaMemcpyAsync(L.bits, p.bits.data(), sizeof(uint32_t) * p.bits.size(), cudaMemcpyHostToDevice,
                                     st));
    ed::centre_kernel<<<1, 256, 0, st>>>(X, cell, p.n, n_rows, d, L.centre);
    ed::prep_kernel<<<(unsigned)ceil_div(p.n, 256), 256, 0, st>>>(X, cell, p.n, n_rows, d, L.status, L.centre,
                                                                   L.offsets, p.G, L.A, L.B, L.group);
    const int64_t chunks = ceil_div(p.n, 32);
    ed::chunk_kernel<<<(unsigned)ceil_div(chunks, 256), 256, 0, st>>>(L.group, L.offsets, p.n, L.chunk);
    RSC_CUDA_TRY(cudaGetLastError());
    if (p.items.empty()) return RSC_OK;
    CUtensorMap ma, mb;
    RSC_CUDA_TRY(tck::make_map(&ma, L.A, p.n, ed::KB, ed::BM));
    RSC_CUDA_TRY(tck::make_map(&mb, L.B, p.n, ed::KB, ed::BN));
    RSC_CUDA_TRY(cudaFuncSetAttribute(ed::edist_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ed::kSmem));
    const int n_items = (int)p.items.size();
    const int grid = std::min(n_items, sm_count());
    ed::edist_tc_kernel<<<grid, ed::kThreads, ed::kSmem, st>>>(ma, mb, L.items, n_items, p.n, L.group, L.offsets,
                                                               L.chunk, p.G, L.bits, S, L.status, tc_wait_budget());
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" {

rsc_status rsc_edistance_workspace_size(int64_t n_rows, int32_t d, const int64_t *group_offsets, int32_t n_groups,
                                        const int32_t *pairs, int64_t n_pairs, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    EdPlan p;
    rsc_status s = plan_edistance(n_rows, d, group_offsets, n_groups, pairs, n_pairs, &p);
    if (s != RSC_OK) return s;
    carve_edistance(nullptr, p, bytes);
    return RSC_OK;
}

rsc_status rsc_edistance(const float *X, int64_t n_rows, int32_t d, const int32_t *cell_index,
                         const int64_t *group_offsets, int32_t n_groups, const int32_t *pairs, int64_t n_pairs,
                         double *sums, double *mean, double *E, void *workspace, size_t workspace_bytes,
                         void *stream) {
    RSC_TRACE("rsc_edistance");
    EdPlan p;
    rsc_status s = plan_edistance(n_rows, d, group_offsets, n_groups, pairs, n_pairs, &p);
    if (s != RSC_OK) return s;
    if (!X || !sums) return fail(RSC_ERR_INVALID_ARG, "X or sums is NULL");
    if (!cell_index && p.n > n_rows) return fail(RSC_ERR_INVALID_ARG, "offsets[G] > n_rows without a cell index");
    size_t need = 0;
    carve_edistance(nullptr, p, &need);
    if (!workspace) return fail(RSC_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(RSC_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, need);
    const EdLayout L = carve_edistance(workspace, p, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = run_edistance_sums(X, n_rows, d, cell_index, group_offsets, p, L, sums, st)) != RSC_OK) return s;
    if (mean || E) {
        const int64_t cells = (int64_t)p.G * p.G;
        ed::assemble_kernel<<<(unsigned)ceil_div(cells, 256), 256, 0, st>>>(sums, L.offsets, p.G, L.bits, mean, E);
        RSC_CUDA_TRY(cudaGetLastError());
    }
    return RSC_OK;
}

}  // extern "C"
