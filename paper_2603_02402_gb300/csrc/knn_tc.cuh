// Tensor-core candidate search kernel, shared by the whole-matrix and the
// batched launches (the work-item policy decides what a CTA scans and
// where it writes).  See knn_tc.cu for the design.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "topk.cuh"

namespace rsc {
namespace tck {


constexpr int BM = 128;              // query rows per item (TMEM lanes)
constexpr int BN = 256;              // database rows per stage = accumulator columns
constexpr int NBUF = 2;              // accumulators (NBUF x BN = 512 TMEM columns); the
                                     // buffer of tile g is g & 1, its phase (g >> 1) & 1
constexpr int QBLK = BM * 128;       // bytes of one 128-row x 64-element bf16 query block
constexpr int DBLK = BN * 128;       // bytes of one 256-row x 64-element bf16 database block
// Operand element size EB: 2 = BF16 (128-byte rows, kind::f16 MMAs of K = 16,
// 128-byte swizzle), 1 = FP8 E4M3 (64-byte rows, kind::f8f6f4 MMAs of K = 32,
// 64-byte swizzle); a 64-element K block is 64 * EB bytes of every row.
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitBudget = 2000000000LL;   // ~1 s of SM clocks: the default budget, and the
                                                  // budget of the drains after a timeout
constexpr uint32_t kSleepNs = 100000;             // suspend limit of one try_wait (ns)
constexpr int kRing = 2;                          // item-index ring slots (dynamic works)

// EG epilogue warpgroups, each owning kCols = BN / EG columns of every tile;
// KCP = top-k list length per (row, part).
template <int KB, int KCP, int EG, int EB = 2>
struct Cfg {
    static constexpr int kCols = BN / EG;
    static constexpr int kEpiThreads = EG * 128;
    static constexpr int kThreads = 64 + kEpiThreads;
    static constexpr int kCap = 24;                                  // buffer entries per thread
    // epilogue that keeps 64 accumulator columns in registers (no re-read on
    // a hit): the shapes whose register budget holds them, for works whose
    // tiles often improve some list (Work::kHitHeavy: the pruned passes; a
    // full scan mostly rejects whole tiles and keeps one vote per tile)
    static constexpr bool kResident = EG == 2 && KCP == 16;
    static constexpr int kQBlk = BM * 64 * EB;    // bytes of one 64-element query K block
    static constexpr int kDBlk = BN * 64 * EB;    // bytes of one 64-element database K block
    static constexpr int kQBytes = KB * kQBlk;
    static constexpr int kStageBytes = KB * kDBlk;
    static constexpr int kBufBytes = kCap * kEpiThreads * 8;
    static constexpr int kBudget = 224 * 1024 - kQBytes - kBufBytes;
    static constexpr int kStages = (kBudget / kStageBytes) > 6 ? 6 : (kBudget / kStageBytes);
    static constexpr int kBarOff = kQBytes + kStages * kStageBytes + kBufBytes;
    static constexpr int kSmem = kBarOff + 256 + 1024;       // barriers + alignment slack
    static_assert(kStages >= 2, "shared memory too small for two stages");
    static_assert(kBarOff % 8 == 0, "barriers 8-byte aligned");
};

// One work item: query rows [q0, q_end) (at most BM) against database rows
// [j_begin, j_end).  short_list: only the best Work::kShort of each list are
// needed (the threshold is the kShort-th key).  A Work with kResume starts
// each (row, part) list from work.resume() instead of empty; one with
// kStartBelow (empty lists, window items whose first tile is the query
// tile's own neighbourhood) starts them below a bound taken from the first
// tile.
struct WorkItem {
    int64_t q0, q_end, j_begin, j_end;
    int tag;
    bool short_list;
    int win_lo, win_hi;     // database tiles [win_lo, win_hi) (counted from j_begin) are scanned first,
    int win_c;              // starting at tile win_c
    const int32_t *tiles;   // non-null: scan exactly these tiles, in this order, nothing else
    int n_tiles;
    bool skip_window;       // scan [0, win_lo) and [win_hi, T) only (the window is already done)
};

// Visiting order of an item's T database tiles: the window [wlo, whi) first,
// from tile c (the query tile's own neighbourhood, so its lists fill with
// near-final values and later tiles insert little): [c, whi), then [wlo, c),
// then [0, wlo), then [whi, T); every tile exactly once.  A tile costs one
// increment and one compare; the range switch runs four times per item.
// Requires 0 <= wlo <= whi <= T.  With an explicit list the tiles are
// lst[0 .. nl) instead, read kAhead entries ahead of use so the list's
// global-memory latency overlaps the tiles in flight (the producer and MMA
// roles; the epilogue, which waits for each accumulator anyway, reads one
// ahead and keeps its registers).
template <int kAhead>
struct TileSeq {
    int m, end, T, wlo, whi, c, phase;
    const int32_t *lst;
    int pos, nl;
    int q[kAhead];   // lst[pos + 1 .. pos + kAhead]

    __device__ __forceinline__ void init(int T_, int wlo_, int whi_, int c_, const int32_t *lst_ = nullptr,
                                         int nl_ = 0, bool skip_window = false) {
        lst = lst_;
        if (lst) {
            pos = 0;
            nl = nl_;
            m = nl > 0 ? lst[0] : 0;
#pragma unroll
            for (int a = 0; a < kAhead; ++a) q[a] = (1 + a < nl) ? lst[1 + a] : 0;
            return;
        }
        T = T_;
        wlo = wlo_;
        whi = whi_;
        c = 0;
        if (skip_window || wlo >= whi) {   // straight to [0, wlo)
            phase = 1;
            m = end = 0;
        } else {
            c = min(max(c_, wlo), whi - 1);
            phase = 0;
            m = c;
            end = whi;
        }
        settle();
    }
    __device__ __forceinline__ void settle() {
        while (m == end && phase < 3) {
            ++phase;
            if (phase == 1) {
                m = wlo;
                end = c;
            } else if (phase == 2) {
                m = 0;
                end = wlo;
            } else {
                m = whi;
                end = T;
            }
        }
    }
    __device__ __forceinline__ bool done() const { return lst ? pos >= nl : m >= end; }
    __device__ __forceinline__ void next() {
        if (lst) {
            ++pos;
            m = q[0];
#pragma unroll
            for (int a = 0; a < kAhead - 1; ++a) q[a] = q[a + 1];
            q[kAhead - 1] = (pos + kAhead < nl) ? lst[pos + kAhead] : 0;
            return;
        }
        if (++m == end) settle();
    }
};

// Position in the ring of S shared-memory stages: stage index and the parity
// of its current round, advanced once per tile (no division in the loop).
struct StageRing {
    int s = 0, S = 2;
    uint32_t ph = 0;
    __device__ __forceinline__ void next() {
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
};

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023);
    return reinterpret_cast<uint8_t *>(a);
}

template <int KB, int KCP, int EG, class Work, int EB = 2>
__global__ void __launch_bounds__(Cfg<KB, KCP, EG, EB>::kThreads, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmD,
              const Work work, unsigned int *status, long long wait_budget, int stages) {
    using C = Cfg<KB, KCP, EG, EB>;
    // pipeline stages in use (the shared-memory layout is sized for C::kStages)
    const int S = (stages >= 2 && stages <= C::kStages) ? stages : C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint8_t *sQ = smem;
    uint8_t *sD = smem + C::kQBytes;
    float *bkey = reinterpret_cast<float *>(sD + S * C::kStageBytes);   // keys, then ids
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::kBarOff);
    uint64_t *full = bars;                     // [S]     database stage loaded
    uint64_t *empty = bars + C::kStages;       // [S]     database stage consumed
    uint64_t *acc_full = bars + 2 * C::kStages;   // [NBUF]  accumulator ready
    uint64_t *acc_empty = acc_full + NBUF;     // [NBUF]  accumulator drained
    uint64_t *q_full = acc_empty + NBUF;
    uint64_t *q_empty = q_full + 1;
    uint64_t *mma_done = q_full + 2;
    uint64_t *item_full = q_full + 3;          // [kRing] next item index published
    uint64_t *item_empty = item_full + kRing;  // [kRing] item index read by every consumer
    volatile int32_t *item_ring = reinterpret_cast<volatile int32_t *>(item_empty + kRing);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(const_cast<int32_t *>(item_ring) + kRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = work.count();

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
        for (int r = 0; r < kRing; ++r) {
            tc::mbar_init(&item_full[r], 1);
            tc::mbar_init(&item_empty[r], 1 + C::kEpiThreads / 32);
        }
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

    // bounded wait: false on timeout (recorded) or when another role aborted;
    // a suspend lasts at most a quarter of the budget (in ns, at least 2
    // clocks per ns), so the budget is checked in time even when it is short
    const uint32_t sleep_ns = (uint32_t)min((long long)kSleepNs, wait_budget / 4);
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
    // Item sequence.  Static works: item blockIdx.x + seq * gridDim.x.
    // Dynamic works (items of very uneven cost): the producer takes the next
    // item from a global counter and publishes it through a kRing-slot ring;
    // the MMA thread and every epilogue warp read the same sequence.  -1 ends
    // it.  Returns false on timeout / abort.
    auto publish_item = [&](int seq, int &it) -> bool {
        if constexpr (!Work::kDynamic) {
            it = blockIdx.x + seq * (int)gridDim.x;
            if (it >= n_items) it = -1;
            return true;
        } else {
            const int r = seq % kRing;
            const uint32_t u = (uint32_t)(seq / kRing);
            if (!wait(&item_empty[r], (u & 1) ^ 1)) return false;
            it = atomicAdd(work.counter, 1);
            if (it >= n_items) it = -1;
            item_ring[r] = it;
            tc::mbar_arrive(&item_full[r]);
            return true;
        }
    };
    auto read_item = [&](int seq, int &it, bool warp_wide) -> bool {
        if constexpr (!Work::kDynamic) {
            it = blockIdx.x + seq * (int)gridDim.x;
            if (it >= n_items) it = -1;
            return true;
        } else {
            const int r = seq % kRing;
            const uint32_t u = (uint32_t)(seq / kRing);
            bool ok_ = wait(&item_full[r], u & 1);
            if (warp_wide) ok_ = __all_sync(0xffffffffu, ok_);
            if (!ok_) return false;
            it = item_ring[r];
            if (warp_wide) __syncwarp();
            if (!warp_wide || (threadIdx.x & 31) == 0) tc::mbar_arrive(&item_empty[r]);
            return true;
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
            StageRing ring;
            ring.S = S;
            int item_no = 0;
            bool ok = true, q_issued = false;
            uint32_t q_parity = 0;
            for (;; ++item_no) {
                int it;
                if (!(ok = publish_item(item_no, it)) || it < 0) break;
                const WorkItem wi = work.get(it);
                const int64_t j_begin = wi.j_begin, j_end = wi.j_end;
                if (!(ok = wait(q_empty, (item_no & 1) ^ 1))) break;
                tc::mbar_arrive_expect_tx(q_full, C::kQBytes);
                for (int kb = 0; kb < KB; ++kb)
                    tc::tma_load_2d(sQ + kb * C::kQBlk, &tmQ, kb * 64, (int)wi.q0, q_full);
                q_issued = true;
                q_parity = item_no & 1;
                const int jb = (int)j_begin, T = (int)((j_end - j_begin + BN - 1) / BN);
                TileSeq<4> sq;
                for (sq.init(T, wi.win_lo, wi.win_hi, wi.win_c, wi.tiles, wi.n_tiles, wi.skip_window); !sq.done();
                     sq.next(), ++gt, ring.next()) {
                    const int s = ring.s;
                    if (!(ok = wait(&empty[s], ring.ph ^ 1u))) break;
                    tc::mbar_arrive_expect_tx(&full[s], C::kStageBytes);
                    const int j0 = jb + sq.m * BN;
                    for (int kb = 0; kb < KB; ++kb)
                        tc::tma_load_2d(sD + (s * KB + kb) * C::kDBlk, &tmD, kb * 64, j0, &full[s]);
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
            constexpr uint32_t idesc = EB == 2 ? tc::idesc_bf16_f32(BM, BN) : tc::idesc_e4m3_f32(BM, BN);
            uint32_t gt = 0;
            StageRing ring;
            ring.S = S;
            int item_no = 0;
            bool ok = true;
            for (;; ++item_no) {
                int it;
                if (!(ok = read_item(item_no, it, false)) || it < 0) break;
                const WorkItem wi = work.get(it);
                const int64_t j_begin = wi.j_begin, j_end = wi.j_end;
                if (!(ok = wait(q_full, item_no & 1))) break;
                tc::tc_fence_after();
                const int T = (int)((j_end - j_begin + BN - 1) / BN);
                TileSeq<4> sq;
                for (sq.init(T, wi.win_lo, wi.win_hi, wi.win_c, wi.tiles, wi.n_tiles, wi.skip_window); !sq.done();
                     sq.next(), ++gt, ring.next()) {
                    const int s = ring.s;
                    const uint32_t b = gt & 1u, v = gt >> 1;
                    if (!(ok = wait(&acc_empty[b], (v & 1) ^ 1))) break;
                    if (!(ok = wait(&full[s], ring.ph))) break;
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + b * BN;
#pragma unroll
                    for (int kb = 0; kb < KB; ++kb) {
                        const uint32_t a_addr = tc::smem_u32(sQ + kb * C::kQBlk);
                        const uint32_t b_addr = tc::smem_u32(sD + (s * KB + kb) * C::kDBlk);
                        if constexpr (EB == 2) {   // four K = 16 steps of 32 bytes in a 128-byte row
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                tc::mma_bf16(d_tmem, tc::smem_desc_sw128(a_addr + kk * 32),
                                             tc::smem_desc_sw128(b_addr + kk * 32), idesc, (kb | kk) != 0);
                            }
                        } else {                   // two K = 32 steps of 32 bytes in a 64-byte row
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                tc::mma_f8(d_tmem, tc::smem_desc_sw64(a_addr + kk * 32),
                                           tc::smem_desc_sw64(b_addr + kk * 32), idesc, (kb | kk) != 0);
                            }
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
        BufferedTopK<KCP, C::kCap, C::kEpiThreads, Work::kShort> tk;
        tk.init(bkey, et);

        const uint32_t tb0 = tmem_base + lane_bits + cbeg;
        uint32_t gt = 0;
        bool ok = true;
        for (int seq = 0;; ++seq) {
            int it;
            if (!(ok = read_item(seq, it, true)) || it < 0) break;
            const WorkItem wi = work.get(it);
            const int jb = (int)wi.j_begin, len = (int)(wi.j_end - wi.j_begin);
            const int T = (len + BN - 1) / BN;
            const int tail = len - (T - 1) * BN;            // columns of the last tile
            const int t_rag = tail < BN ? T - 1 : -1;       // the last tile, when it is partial
            tk.reset();
            tk.shortl = wi.short_list;
            if constexpr (Work::kResume) {   // continue lists saved by an earlier pass
                const int64_t q = wi.q0 + r;
                if (q < wi.q_end) work.template resume<EG>(wi, part, q, tk.list);
            }
            TileSeq<1> sq;
            bool first = Work::kStartBelow;   // the item's first tile, lists still empty
            for (sq.init(T, wi.win_lo, wi.win_hi, wi.win_c, wi.tiles, wi.n_tiles, wi.skip_window); !sq.done();
                 sq.next(), ++gt, first = false) {
                const uint32_t b = gt & 1u;
                ok = wait(&acc_full[b], (gt >> 1) & 1u);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t tb = tb0 + b * BN;
                const bool rag = sq.m == t_rag;
                const int j0 = jb + sq.m * BN + cbeg;
                const int valid = rag ? tail - cbeg : C::kCols;
                if (Work::kStartBelow && first && !rag) {
                    // first tile of empty lists: the largest of the kCols / 8
                    // minima of 8 columns bounds the KCP-th smallest value from
                    // above (kCols / 8 >= KCP distinct values lie at or below
                    // it), so the lists start from that bound instead of +inf
                    // and never take the larger values in
                    float gmax = -INFINITY;
#pragma unroll 1
                    for (int c0 = 0; c0 < C::kCols; c0 += 32) {
                        float vv[32];
                        __syncwarp();
                        tc::tmem_ld32(tb + c0, vv);
                        tc::tmem_wait_ld();
                        float g[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) g[h] = min8(vv + 8 * h);
                        gmax = fmaxf(gmax, fmaxf(fmaxf(g[0], g[1]), fmaxf(g[2], g[3])));
                    }
                    if constexpr (C::kCols / 8 >= KCP) tk.start_below(gmax);
                }
                if constexpr (C::kResident && Work::kHitHeavy) {
                    // 64 columns at a time held in registers: minima of 8, one
                    // vote on their minimum, offers straight from the registers
#pragma unroll 1
                    for (int c0 = 0; c0 < C::kCols; c0 += 64) {
                        float va[32], vb[32];
                        __syncwarp();
                        tc::tmem_ld32(tb + c0, va);
                        tc::tmem_ld32(tb + c0 + 32, vb);
                        tc::tmem_wait_ld();
                        if (valid < c0 + 64) {   // ragged end of the range (warp-uniform)
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                if (c0 + i >= valid) va[i] = INFINITY;
                                if (c0 + 32 + i >= valid) vb[i] = INFINITY;
                            }
                        }
                        float m8[8];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            m8[h] = min8(va + 8 * h);
                            m8[4 + h] = min8(vb + 8 * h);
                        }
                        const float m64 = fminf(fmin3(fmin3(m8[0], m8[1], m8[2]), fmin3(m8[3], m8[4], m8[5]), m8[6]),
                                                m8[7]);
                        if (__any_sync(0xffffffffu, m64 < tk.bound())) {
                            tk.offer16m(va, m8[0], m8[1], j0 + c0);
                            tk.offer16m(va + 16, m8[2], m8[3], j0 + c0 + 16);
                            tk.offer16m(vb, m8[4], m8[5], j0 + c0 + 32);
                            tk.offer16m(vb + 16, m8[6], m8[7], j0 + c0 + 48);
                        }
                    }
                } else if constexpr (KCP >= 64) {
                    // long lists leave little register room: 16 columns per load
                    float mn = INFINITY;
#pragma unroll 1
                    for (int c0 = 0; c0 < C::kCols; c0 += 16) {
                        float vv[16];
                        __syncwarp();
                        tc::tmem_ld16(tb + c0, vv);
                        tc::tmem_wait_ld();
                        mn = fminf(mn, min_of(vv));
                    }
                    if (__any_sync(0xffffffffu, rag || mn < tk.bound())) {
#pragma unroll 1
                        for (int c0 = 0; c0 < C::kCols; c0 += 16) {
                            float vv[16];
                            __syncwarp();
                            tc::tmem_ld16(tb + c0, vv);
                            tc::tmem_wait_ld();
                            if (valid < c0 + 16) {   // ragged end of the range (warp-uniform)
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    if (c0 + i >= valid) vv[i] = INFINITY;
                            }
                            tk.offer16(vv, j0 + c0);
                        }
                    }
                } else {
                    // fast path: minimum of this thread's kCols values, one vote per tile
                    float mn = INFINITY;
#pragma unroll 1
                    for (int c0 = 0; c0 < C::kCols; c0 += 32) {
                        float vv[32];
                        __syncwarp();
                        tc::tmem_ld32(tb + c0, vv);
                        tc::tmem_wait_ld();
                        mn = fminf(mn, min_of(vv));
                    }
                    if (__any_sync(0xffffffffu, rag || mn < tk.bound())) {
                        // some lane may improve its list (or the tile is partial):
                        // read the accumulator again and offer every value
#pragma unroll 1
                        for (int c0 = 0; c0 < C::kCols; c0 += 32) {
                            float vv[32];
                            __syncwarp();
                            tc::tmem_ld32(tb + c0, vv);
                            tc::tmem_wait_ld();
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
                            tk.offer16(lo, j0 + c0);
                            tk.offer16(hi, j0 + c0 + 16);
                        }
                    }
                }
                // hand the accumulator part back to the MMA warp
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
            }
            if (!ok) break;
            tk.flush();
            const int64_t q = wi.q0 + r;
            if (q < wi.q_end) work.template emit<EG>(wi, part, q, tk.list);
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

// Whole-matrix work: query tile qt (BM rows) x database split sp.
struct PlainWork {
    static constexpr int kShort = 0;   // never used (short_list is false)
    static constexpr bool kResume = false;
    static constexpr bool kHitHeavy = false;
    static constexpr bool kStartBelow = false;
    static constexpr bool kDynamic = false;
    int64_t n;
    int splits;
    int64_t split_len;
    int32_t *cand;    // [splits * EG, n, KCP]
    int n_items;
    int window;       // tiles on either side of the query tile scanned first (0: none)

    int64_t count_host() const { return n_items; }
    __device__ __forceinline__ int count() const { return n_items; }
    __device__ __forceinline__ WorkItem get(int it) const {
        const int qt = it / splits, sp = it - qt * splits;
        WorkItem w;
        w.q0 = (int64_t)qt * BM;
        w.q_end = min(n, w.q0 + BM);
        w.j_begin = (int64_t)sp * split_len;
        w.j_end = min(n, w.j_begin + split_len);
        w.tag = sp;
        w.short_list = false;
        w.win_lo = w.win_hi = w.win_c = 0;
        w.tiles = nullptr;
        w.n_tiles = 0;
        w.skip_window = false;
        if (window > 0 && w.q0 >= w.j_begin && w.q0 < w.j_end) {
            const int T = (int)((w.j_end - w.j_begin + BN - 1) / BN);
            const int tq = (int)((w.q0 - w.j_begin) / BN);
            w.win_lo = max(0, tq - window);
            w.win_hi = min(T, tq + window + 1);
            w.win_c = tq;
        }
        return w;
    }
    template <int EG, int KCP>
    __device__ __forceinline__ void emit(const WorkItem &w, int part, int64_t q, const RowTopK<KCP> &list) const {
        int32_t *out = cand + ((int64_t)(w.tag * EG + part) * n + q) * KCP;
#pragma unroll
        for (int c = 0; c < KCP; ++c) out[c] = list.id[c];
    }
};

template <int KB, int KCP, int EG, class Work, int EB = 2>
cudaError_t launch_kernel(const CUtensorMap &mq, const CUtensorMap &md, const Work &work, unsigned int *status,
                          cudaStream_t st, int stages = 0) {
    using C = Cfg<KB, KCP, EG, EB>;
    auto kern = knn_tc_kernel<KB, KCP, EG, Work, EB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    const int64_t items = work.count_host();
    if (items <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(items, sm_count());
    kern<<<grid, C::kThreads, C::kSmem, st>>>(mq, md, work, status, tc_wait_budget(), stages);
    return cudaGetLastError();
}

cudaError_t make_map(CUtensorMap *m, const void *base, int64_t rows, int KB, int box_rows);
// [rows, 64] FP8 bytes, box_rows x 64-byte boxes, 64-byte swizzle
cudaError_t make_map_fp8(CUtensorMap *m, const void *base, int64_t rows, int box_rows);

}  // namespace tck
}  // namespace rsc
