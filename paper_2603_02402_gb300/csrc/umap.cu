// UMAP layout on the fuzzy graph: epochs of edge-sampled stochastic gradient
// moves (the UMAP method's embedding optimisation, which the paper runs on
// the neighbourhood graph: Methods, "Dimensionality reduction and graph
// analysis").  phi(d) = 1 / (1 + a d^(2b)); a sampled entry i -> j pulls its
// endpoints together along the gradient of log phi and draws `r` vertices
// uniformly that push i away along the gradient of gamma log(1 - phi) (squared
// distance offset by 0.001); every coordinate of a move is clipped to [-4, 4]
// and scaled by alpha_n = lr (1 - (n - 1) / N).  Entry e is sampled in epoch n
// when floor(n f_e) > floor((n - 1) f_e), f_e = w_e / max w (single
// precision), and negative q of entry e in epoch n is vertex h * n >> 32,
// h the high (q even) or low (q odd) 32 bits of SplitMix64 output number
// ((n - 1) nnz + e) ceil(r / 2) + floor(q / 2) + 1.
//
// An epoch reads the positions it started with and writes new ones (two
// buffers), so its result does not depend on the order threads run in.  On a
// symmetric graph (G_ij == G_ji, both entries stored, as the fuzzy union is)
// the entries i -> j and j -> i are sampled in the same epochs, and the
// attraction vertex i receives from both is 2 alpha clip(c (y_i - y_j)): each
// row gathers its own moves, so no vertex is written by two warps and no
// atomics are needed.  A warp owns 32 consecutive rows: it streams their
// entries (sampling frequency, column and a byte holding the entry's row
// inside the block), queues the sampled ones in shared memory, and works
// through the queue in batches of 32 entries, one per lane, each lane loading
// its 1 + r positions together; a segmented scan over the lanes adds each
// row's share in a fixed order.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

constexpr int kUmapWarps = 2;   // warps per block (each owns kRowsPerWarp rows)

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;   // SplitMix64 state increment

// SplitMix64 output for state z (= seed + i * kGolden for output number i).
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Hardware approximations (PTX lg2 / ex2 / rcp .approx.ftz): log2 with an
// absolute error near 2^-22, which is what the power 2^(b log2 x) needs.
__device__ __forceinline__ float lg2_fast(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float clip4(float v) { return fminf(fmaxf(v, -4.f), 4.f); }

// Largest weight (NaN and non-positive weights ignored) into *wmax (bits of a
// non-negative float, atomicMax on the integer order).
__global__ void __launch_bounds__(256) umap_wmax_kernel(const float *__restrict__ data, int64_t nnz,
                                                        unsigned int *wmax_bits) {
    float m = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, data[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(wmax_bits, __float_as_uint(m));
}

// f_e = w_e / max w (IEEE division), 0 when no weight is positive.
__global__ void __launch_bounds__(256) umap_freq_kernel(const float *__restrict__ data, int64_t nnz,
                                                        const unsigned int *__restrict__ wmax_bits,
                                                        float *__restrict__ f) {
    const float wmax = __uint_as_float(*wmax_bits);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        f[e] = wmax > 0.f ? __fdiv_rn(data[e], wmax) : 0.f;
}

// rowoff[e] = (row of entry e) mod 32, the entry's row inside its warp's block
// of 32 rows (warp per row; entries outside [0, nnz) are not written).
__global__ void __launch_bounds__(256) umap_rowoff_kernel(const int64_t *__restrict__ indptr, int64_t n, int64_t nnz,
                                                          uint8_t *__restrict__ rowoff) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int64_t beg = std::max(indptr[i], (int64_t)0), end = std::min(indptr[i + 1], nnz);
    for (int64_t e = beg + (threadIdx.x & 31); e < end; e += 32) rowoff[e] = (uint8_t)(i & 31);
}

// Embedding [n, D] (caller's layout) <-> internal rows of DS floats.
template <int D, int DS>
__global__ void __launch_bounds__(256) umap_pack_kernel(const float *__restrict__ src, int64_t n,
                                                        float *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int t = 0; t < DS; ++t) dst[i * DS + t] = t < D ? src[i * D + t] : 0.f;
}

template <int D, int DS>
__global__ void __launch_bounds__(256) umap_unpack_kernel(const float *__restrict__ src, int64_t n,
                                                          float *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int t = 0; t < D; ++t) dst[i * D + t] = src[i * DS + t];
}

template <int DS>
struct Vec {
    float v[DS];
};

template <int D, int DS>
__device__ __forceinline__ Vec<DS> load_row(const float *__restrict__ Y, int i) {
    Vec<DS> r;
    if constexpr (DS == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(Y) + i);
        r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else if constexpr (DS == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(Y) + i);
        r.v[0] = q.x; r.v[1] = q.y;
    } else {
        r.v[0] = __ldg(Y + i);
    }
    return r;
}

// Rows per warp: a warp owns the moves of 32 consecutive rows.
constexpr int kRowsPerWarp = 32;
// Entry chunks (32 entries each) whose f and columns are loaded together.
constexpr int kChunkGroup = 4;
// Queue of sampled entries: a batch of 32 plus one group's worth.
constexpr int kQueue = 32 + 32 * kChunkGroup;
// Negative samples whose positions are loaded together.
constexpr int kNegGroup = 8;

struct UmapWarpSmem {
    float acc[kRowsPerWarp][4];      // moves gathered per row
    float y[kRowsPerWarp][4];        // the rows' own positions
    int32_t qe[kQueue];              // queue of sampled entries: entry index
    int32_t qj[kQueue];              //   its column
    int32_t qr[kQueue];              //   its row inside the warp's block
};

// Moves of a batch: lane L takes queued entry off + L (L < cnt) and returns
// its attraction (doubled, for the mirror entry) plus its negatives' repulsion.
template <int D, int DS>
__device__ __forceinline__ void batch_moves(const UmapWarpSmem &sm, int lane, int off, int cnt, int64_t r0,
                                            const float *__restrict__ Yin, int64_t n, int64_t nnz, int epoch,
                                            const UmapParams &p, float alpha, float (&acc)[D]) {
#pragma unroll
    for (int t = 0; t < D; ++t) acc[t] = 0.f;
    if (lane >= cnt) return;
    const int64_t e = sm.qe[off + lane];
    // negatives 2h and 2h + 1 take the high and low halves of output number
    // ((n - 1) nnz + e) ceil(r / 2) + h + 1 (state seed + number * kGolden)
    const uint64_t ctr0 = ((uint64_t)(epoch - 1) * (uint64_t)nnz + (uint64_t)e) * (uint64_t)((p.neg_rate + 1) >> 1);
    uint64_t state = p.seed + (ctr0 + 1) * kGolden;
    Vec<DS> yi;
    const int row = sm.qr[off + lane];
#pragma unroll
    for (int t = 0; t < DS; ++t) yi.v[t] = sm.y[row][t];
    const Vec<DS> yj = load_row<D, DS>(Yin, sm.qj[off + lane]);
    const float gb2 = 2.f * p.gamma * p.b;
#pragma unroll 1
    for (int q0 = 0; q0 < max(p.neg_rate, 1); q0 += kNegGroup) {   // one pass at least, for the attraction
        Vec<DS> yv[kNegGroup];
#pragma unroll
        for (int g = 0; g < kNegGroup; g += 2) {
            if (q0 + g < p.neg_rate) {
                const uint64_t r64 = splitmix64_mix(state);
                state += kGolden;
                yv[g] = load_row<D, DS>(Yin, (int)__umulhi((unsigned int)(r64 >> 32), (unsigned int)n));
                if (q0 + g + 1 < p.neg_rate)
                    yv[g + 1] = load_row<D, DS>(Yin, (int)__umulhi((unsigned int)r64, (unsigned int)n));
            }
        }
        if (q0 == 0) {   // attraction: c = -2ab d2^(b-1) / (1 + a d2^b)
            float dy[D], d2 = 0.f;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                dy[t] = yi.v[t] - yj.v[t];
                d2 = fmaf(dy[t], dy[t], d2);
            }
            if (d2 > 0.f) {
                const float lg = lg2_fast(d2);
                const float pb = ex2_fast(p.b * lg), pbm1 = ex2_fast((p.b - 1.f) * lg);
                const float c = -2.f * p.a * p.b * pbm1 * rcp_fast(fmaf(p.a, pb, 1.f));
                const float s = 2.f * alpha;   // entry i -> j and its mirror j -> i
#pragma unroll
                for (int t = 0; t < D; ++t) acc[t] = fmaf(s, clip4(c * dy[t]), acc[t]);
            }
        }
        // repulsion: c = 2 gamma b / ((0.001 + d2)(1 + a d2^b))
#pragma unroll
        for (int g = 0; g < kNegGroup; ++g) {
            if (q0 + g >= p.neg_rate) break;
            float dy[D], d2 = 0.f;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                dy[t] = yi.v[t] - yv[g].v[t];
                d2 = fmaf(dy[t], dy[t], d2);
            }
            if (d2 > 0.f) {
                const float pb = ex2_fast(p.b * lg2_fast(d2));
                const float c = gb2 * rcp_fast((0.001f + d2) * fmaf(p.a, pb, 1.f));
#pragma unroll
                for (int t = 0; t < D; ++t) acc[t] = fmaf(alpha, clip4(c * dy[t]), acc[t]);
            }
        }
    }
}

// Adds each row's share of a batch to sm.acc: a segmented inclusive scan over
// the lanes (queued entries are in row order), then the last lane of every
// row's segment adds the row's sum.  The order of additions depends only on
// the queue, so the epoch is deterministic.
template <int D>
__device__ __forceinline__ void batch_reduce(UmapWarpSmem &sm, int lane, int off, int cnt, float (&acc)[D]) {
    const int row = lane < cnt ? sm.qr[off + lane] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ro = __shfl_up_sync(0xffffffffu, row, o);
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const float v = __shfl_up_sync(0xffffffffu, acc[t], o);
            if (lane >= o && ro == row) acc[t] += v;
        }
    }
    const int rn = __shfl_down_sync(0xffffffffu, row, 1);
    if (lane < cnt && (lane == cnt - 1 || rn != row)) {
#pragma unroll
        for (int t = 0; t < D; ++t) sm.acc[row][t] += acc[t];
    }
    __syncwarp();
}

// One epoch: warp per 32 rows.  The warp streams its rows' entries in groups
// of kChunkGroup x 32 (f and columns loaded together), queues the sampled
// ones, and works through the queue in batches of 32 entries, one per lane,
// each lane loading its 1 + r positions together.
template <int D, int DS>
__global__ void __launch_bounds__(32 * kUmapWarps)
umap_epoch_kernel(const int64_t *__restrict__ indptr, const int32_t *__restrict__ indices,
                  const float *__restrict__ f, const uint8_t *__restrict__ rowoff, int64_t n, int64_t nnz,
                  const float *__restrict__ Yin, float *__restrict__ Yout, int epoch, UmapParams p,
                  unsigned int *status) {
    __shared__ UmapWarpSmem smem[kUmapWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    UmapWarpSmem &sm = smem[warp];
    const int64_t r0 = ((int64_t)blockIdx.x * kUmapWarps + warp) * kRowsPerWarp;
    if (r0 >= n) return;
    const int rows = (int)std::min<int64_t>(kRowsPerWarp, n - r0);
    // Row boundaries 0 .. rows, made monotone inside [0, nnz] (a bad indptr
    // is recorded and its rows shrink; nothing outside the arrays is read).
    int64_t b = indptr[r0 + std::min(lane, rows)];
    const int64_t b_last = indptr[r0 + rows];
    bool bad = lane <= rows && (b < 0 || b > nnz);
    b = lane <= rows ? std::min(std::max(b, (int64_t)0), nnz) : nnz;
    int64_t m = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, m, o);
        if (lane >= o) m = std::max(m, v);
    }
    bad |= lane <= rows && m != b;
    const int64_t prev = __shfl_sync(0xffffffffu, m, rows - 1);
    const int64_t last = std::max(std::min(std::max(b_last, (int64_t)0), nnz), prev);
    bad |= lane == 0 && (b_last < 0 || b_last > nnz || b_last < prev);
    if (__any_sync(0xffffffffu, bad) && lane == 0) record_status(status, RSC_ERR_INVALID_ARG);
#pragma unroll
    for (int t = 0; t < 4; ++t) (&sm.acc[0][0])[t * 32 + lane] = 0.f;
    if (lane < rows) {
        const Vec<DS> y = load_row<D, DS>(Yin, (int)r0 + lane);
#pragma unroll
        for (int t = 0; t < DS; ++t) sm.y[lane][t] = y.v[t];
    }
    __syncwarp();
    const int64_t E1 = last;
    const float now = (float)epoch, before = (float)(epoch - 1);
    const float alpha = p.lr * (1.f - (float)(epoch - 1) / (float)p.n_epochs);
    int64_t base = __shfl_sync(0xffffffffu, m, 0);
    int qc = 0;   // queued entries
    float acc[D];
    while (true) {
        const bool more = base < E1;
        if (more) {
            float fe[kChunkGroup];
            int32_t col[kChunkGroup];
            int ro[kChunkGroup];
#pragma unroll
            for (int g = 0; g < kChunkGroup; ++g) {
                const int64_t e = base + 32 * g + lane;
                fe[g] = e < E1 ? f[e] : 0.f;
                col[g] = e < E1 ? indices[e] : 0;
                ro[g] = e < E1 ? rowoff[e] : 0;
            }
            unsigned int mk[kChunkGroup];
#pragma unroll
            for (int g = 0; g < kChunkGroup; ++g) {
                const int64_t e = base + 32 * g + lane;
                bool take = e < E1 && floorf(__fmul_rn(now, fe[g])) > floorf(__fmul_rn(before, fe[g]));
                if (take && (col[g] < 0 || (int64_t)col[g] >= n)) {
                    record_status(status, RSC_ERR_INVALID_ARG);
                    take = false;
                }
                mk[g] = __ballot_sync(0xffffffffu, take);
            }
#pragma unroll
            for (int g = 0; g < kChunkGroup; ++g) {
                if ((mk[g] >> lane) & 1u) {
                    const int slot = qc + __popc(mk[g] & ((1u << lane) - 1u));
                    sm.qe[slot] = (int32_t)(base + 32 * g + lane);
                    sm.qj[slot] = col[g];
                    sm.qr[slot] = min(ro[g], rows - 1);   // a bad indptr can leave stale bytes: stay in the block
                }
                qc += __popc(mk[g]);
            }
            base += 32 * kChunkGroup;
            __syncwarp();
        }
        // Full batches; at the end also the last partial one.
        int done = 0;
        while (qc - done >= 32 || (!more && qc > done)) {
            const int cnt = min(32, qc - done);
            batch_moves<D, DS>(sm, lane, done, cnt, r0, Yin, n, nnz, epoch, p, alpha, acc);
            batch_reduce<D>(sm, lane, done, cnt, acc);
            done += cnt;
        }
        if (done > 0) {   // move the rest (< 32) to the front
            const int rest = qc - done;
            int32_t e_ = 0, j_ = 0, r_ = 0;
            if (lane < rest) {
                e_ = sm.qe[done + lane];
                j_ = sm.qj[done + lane];
                r_ = sm.qr[done + lane];
            }
            __syncwarp();
            if (lane < rest) {
                sm.qe[lane] = e_;
                sm.qj[lane] = j_;
                sm.qr[lane] = r_;
            }
            qc = rest;
            __syncwarp();
        }
        if (!more) break;
    }
    if (lane < rows) {
#pragma unroll
        for (int t = 0; t < DS; ++t) Yout[(r0 + lane) * DS + t] = t < D ? sm.y[lane][t] + sm.acc[lane][t] : 0.f;
    }
}

template <int D, int DS>
cudaError_t run_epochs(const int64_t *indptr, const int32_t *indices, const float *f, const uint8_t *rowoff,
                       int64_t n, int64_t nnz, float *embedding, float *buf0, float *buf1, int first, int last,
                       UmapParams p, unsigned int *status, cudaStream_t st) {
    const unsigned pb = (unsigned)ceil_div(n, 256);
    umap_pack_kernel<D, DS><<<pb, 256, 0, st>>>(embedding, n, buf0);
    const unsigned eb = (unsigned)ceil_div(n, (int64_t)kUmapWarps * kRowsPerWarp);
    float *src = buf0, *dst = buf1;
    for (int epoch = first; epoch <= last; ++epoch) {
        umap_epoch_kernel<D, DS><<<eb, 32 * kUmapWarps, 0, st>>>(indptr, indices, f, rowoff, n, nnz, src, dst, epoch,
                                                                   p, status);
        float *t = src;
        src = dst;
        dst = t;
    }
    umap_unpack_kernel<D, DS><<<pb, 256, 0, st>>>(src, n, embedding);
    return cudaGetLastError();
}

}  // namespace

int umap_row_floats(int dim) { return dim == 3 ? 4 : dim; }

cudaError_t launch_umap_prepare(const int64_t *indptr, const float *data, int64_t n, int64_t nnz,
                                unsigned int *wmax_bits, float *f, uint8_t *rowoff, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(wmax_bits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess || nnz == 0) return e;
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(nnz, 256), (int64_t)sm_count() * 8);
    umap_wmax_kernel<<<g, 256, 0, st>>>(data, nnz, wmax_bits);
    umap_freq_kernel<<<g, 256, 0, st>>>(data, nnz, wmax_bits, f);
    umap_rowoff_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, st>>>(indptr, n, nnz, rowoff);
    return cudaGetLastError();
}

cudaError_t launch_umap_epochs(const int64_t *indptr, const int32_t *indices, const float *f, const uint8_t *rowoff,
                               int64_t n, int64_t nnz, int dim, float *embedding, float *buf0, float *buf1, int first,
                               int last, UmapParams p, unsigned int *status, cudaStream_t st) {
#define RSC_UMAP_CASE(D, DS) \
    return run_epochs<D, DS>(indptr, indices, f, rowoff, n, nnz, embedding, buf0, buf1, first, last, p, status, st)
    switch (dim) {
        case 1: RSC_UMAP_CASE(1, 1);
        case 2: RSC_UMAP_CASE(2, 2);
        case 3: RSC_UMAP_CASE(3, 4);
        case 4: RSC_UMAP_CASE(4, 4);
        default: return cudaErrorInvalidValue;
    }
#undef RSC_UMAP_CASE
}

}  // namespace rsc
