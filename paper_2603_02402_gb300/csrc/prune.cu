// Tile pruning bounds for the tensor-core search (rows in locality order).
//
// The accumulator of query row i and database row j holds, up to the
// tensor core's FP32 accumulation error e_ij,
//     acc_ij = |v_i - v_j|^2 - |v_i|^2 - beta |v_j|^2,
// where v are the BF16-rounded operand rows (Euclidean: the centred row,
// beta = 0, the |v_j|^2 term being folded into the MMA; cosine: the
// normalised row plus its zero-row flag, beta = 1).  A list of row i accepts
// acc_ij only below its threshold thr_i, i.e. only when
//     |v_i - v_j|^2 < thr_i + |v_i|^2 + beta |v_j|^2 + e_ij.
// With spheres (c_Q, r_Q) around the query tile's v and (c_t, r_t) around
// database tile t's v, |v_i - v_j| >= |c_Q - c_t| - r_Q - r_t for every pair,
// so tile t can be dropped for query tile Q when
//     (|c_Q - c_t| - r_Q - r_t)^2 - beta N_t - margin > tau_Q,
// tau_Q = max over the tile's rows and parts of (thr + |v_i|^2), N_t =
// max |v_j|^2 over t, and margin bounds e_ij and the FP32 rounding of these
// bounds: 2^-11 (N_Q + N_t), sixteen times the worst-case error of a K = 64
// FP32 accumulation of terms summing to at most 2 (N_Q + N_t) in magnitude.
// Radii are inflated by 2^-10 relative plus 1e-6 for their own rounding.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace rsc {

namespace {

constexpr int kCen = 64;           // centre stride (floats); v has at most 64 components
constexpr int kChunkTiles = 256;   // database tiles per block in the bound passes
constexpr int kBoundThreads = 128; // query tiles per block in the bound passes
constexpr int kStage = 32;         // database tiles staged in shared memory at once
constexpr int kGroupTiles = 16;    // database tiles per group sphere (tested before its tiles)

// Warp per group of rows of the BF16 query operand (row stride W elements,
// v = the first dv <= 64 of them): rows [g * R, (g + 1) * R) clipped to n, or
// [g_start[g], g_end[g]) when given.  Centre (mean of v), radius (max |v - c|,
// inflated), max |v|^2; row_norm[i] = |v_i|^2 when requested.
// Lane l reads 16 bytes (components 8 (l & 7) .. + 7) of row l >> 3 of every
// 4-row step, so a warp moves four 128-byte rows per load and keeps several
// steps in flight; the 8 lanes of a row combine by shuffles.  The centre is
// any point (its rounding does not matter); the radius is measured from it.
__global__ void tile_sphere_kernel(const uint16_t *__restrict__ Qb, int64_t n, int W, int dv, int R, int groups,
                                   const int64_t *__restrict__ g_start, const int64_t *__restrict__ g_end,
                                   float *__restrict__ cen, float *__restrict__ rad, float *__restrict__ nmax,
                                   float *__restrict__ row_norm) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= groups) return;
    const int64_t r0 = g_start ? g_start[g] : (int64_t)g * R;
    const int64_t r1 = g_end ? g_end[g] : min(n, r0 + R);
    const int ch = lane & 7, rs = lane >> 3;
    int nv = dv - 8 * ch;   // valid components of this lane's 8
    nv = nv < 0 ? 0 : (nv > 8 ? 8 : nv);
    auto load = [&](int64_t r, float (&v)[8]) {
        const uint4 u = *reinterpret_cast<const uint4 *>(Qb + r * W + 8 * ch);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = 2 * i < nv ? __uint_as_float(w4[i] << 16) : 0.f;
            v[2 * i + 1] = 2 * i + 1 < nv ? __uint_as_float(w4[i] & 0xffff0000u) : 0.f;
        }
    };
    float c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = 0.f;
#pragma unroll 4
    for (int64_t r = r0 + rs; r < r1; r += 4) {
        float v[8];
        load(r, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] += v[i];
    }
    const float inv = 1.f / (float)(r1 - r0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i] += __shfl_xor_sync(0xffffffffu, c[i], 8);
        c[i] += __shfl_xor_sync(0xffffffffu, c[i], 16);
        c[i] *= inv;
    }
    float md = 0.f, mn = 0.f;
    // rows of the last, partial step: lanes past r1 contribute nothing but
    // still take part in the shuffles
    for (int64_t base = r0; base < r1; base += 4) {
        const int64_t r = base + rs;
        const bool ok = r < r1;
        float v[8];
        if (ok) load(r, v);
        float dd = 0.f, nn = 0.f;
        if (ok) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float e = v[i] - c[i];
                dd = fmaf(e, e, dd);
                nn = fmaf(v[i], v[i], nn);
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            dd += __shfl_xor_sync(0xffffffffu, dd, o);
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
        }
        md = fmaxf(md, dd);
        mn = fmaxf(mn, nn);
        if (row_norm && ok && ch == 0) row_norm[r] = nn;
    }
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, 8));
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, 16));
    mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, 8));
    mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, 16));
    if (rs == 0) {
        float4 *out = reinterpret_cast<float4 *>(cen + (int64_t)g * kCen + 8 * ch);
        out[0] = make_float4(c[0], c[1], c[2], c[3]);
        out[1] = make_float4(c[4], c[5], c[6], c[7]);
    }
    if (lane == 0) {
        rad[g] = sqrtf(md) * (1.f + 0x1p-10f) + 1e-6f;
        nmax[g] = mn;
    }
}

// tau_Q = max over the query tile's rows and parts of (saved threshold +
// |v_i|^2); infinite while some list is not full.  Warp per query tile.
__global__ void tile_tau_kernel(const float *__restrict__ st_key, int64_t n, int EG, int KCP,
                                const float *__restrict__ row_norm, int qtiles, int BM, float *__restrict__ tau) {
    const int qt = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qt >= qtiles) return;
    float m = -INFINITY;
    const int64_t r0 = (int64_t)qt * BM, r1 = min(n, r0 + BM);
    for (int64_t q = r0 + lane; q < r1; q += 32)
        for (int p = 0; p < EG; ++p) m = fmaxf(m, st_key[(q * EG + p) * KCP + KCP - 1] + row_norm[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) tau[qt] = m;
}

// Spheres around groups of kGroupTiles consecutive database tiles, from the
// tiles' own spheres: centre = mean of the tile centres, radius = max over
// the tiles of |c_G - c_t| + r_t (inflated), max norm = max over the tiles.
// Every row of the group lies inside it, so a group that fails the drop test
// for a query tile drops each of its tiles.  Warp per group.
__global__ void group_sphere_kernel(const float *__restrict__ dcen, const float *__restrict__ drad,
                                    const float *__restrict__ dn, int dtiles, int groups, float *__restrict__ gcen,
                                    float *__restrict__ grad, float *__restrict__ gn) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= groups) return;
    const int t0 = g * kGroupTiles, t1 = min(dtiles, t0 + kGroupTiles);
    float c0 = 0.f, c1 = 0.f;
    for (int t = t0; t < t1; ++t) {
        c0 += dcen[(int64_t)t * kCen + lane];
        c1 += dcen[(int64_t)t * kCen + lane + 32];
    }
    const float inv = 1.f / (float)(t1 - t0);
    c0 *= inv;
    c1 *= inv;
    float r = 0.f, m = 0.f;
    for (int t = t0; t < t1; ++t) {
        const float e0 = dcen[(int64_t)t * kCen + lane] - c0, e1 = dcen[(int64_t)t * kCen + lane + 32] - c1;
        float dd = e0 * e0 + e1 * e1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
        r = fmaxf(r, sqrtf(dd) * (1.f + 0x1p-10f) + drad[t]);
        m = fmaxf(m, dn[t]);
    }
    gcen[(int64_t)g * kCen + lane] = c0;
    gcen[(int64_t)g * kCen + lane + 32] = c1;
    if (lane == 0) {
        grad[g] = r * (1.f + 0x1p-10f) + 1e-6f;
        gn[g] = m;
    }
}

// Drop test of a database sphere (centre sc, radius r, max norm nt) for the
// query tile with centre c, radius rq, max norm nq and threshold tq.
__device__ __forceinline__ bool sphere_drop(const float (&c)[kCen], const float *sc, float r, float nt, float rq,
                                            float nq, float tq, float beta) {
    const float4 *dc = reinterpret_cast<const float4 *>(sc);
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int u = 0; u < kCen / 4; u += 2) {
        const float4 x = dc[u], y = dc[u + 1];
        float f;
        f = c[4 * u] - x.x; a0 = fmaf(f, f, a0);
        f = c[4 * u + 1] - x.y; a0 = fmaf(f, f, a0);
        f = c[4 * u + 2] - x.z; a0 = fmaf(f, f, a0);
        f = c[4 * u + 3] - x.w; a0 = fmaf(f, f, a0);
        f = c[4 * u + 4] - y.x; a1 = fmaf(f, f, a1);
        f = c[4 * u + 5] - y.y; a1 = fmaf(f, f, a1);
        f = c[4 * u + 6] - y.z; a1 = fmaf(f, f, a1);
        f = c[4 * u + 7] - y.w; a1 = fmaf(f, f, a1);
    }
    const float gap = sqrtf(a0 + a1) - rq - r;
    const float margin = 0x1p-11f * (nq + nt);
    return gap > 0.f && gap * gap - beta * nt - margin > tq;
}

// Thread per query tile Q, block column = a chunk of kChunkTiles database
// tiles: count the kept tiles of (Q, chunk) and record them as bits, one
// 32-bit word per stage of kStage tiles (bits[(Q * nchunk + chunk) * kWords
// + stage]).  Each group of kGroupTiles tiles is tested first: a query tile
// that drops the group skips its tiles (each of them would be dropped too).
constexpr int kWords = kChunkTiles / kStage;
static_assert(kStage == 32, "one bit word per stage");

__global__ void __launch_bounds__(kBoundThreads)
prune_tiles_kernel(int qtiles, int dtiles, int nchunk, int qpt, int window, float beta,
                   const float *__restrict__ qcen, const float *__restrict__ qrad, const float *__restrict__ qn,
                   const float *__restrict__ tau, const float *__restrict__ dcen, const float *__restrict__ drad,
                   const float *__restrict__ dn, const float *__restrict__ gcen, const float *__restrict__ grad,
                   const float *__restrict__ gn, int32_t *__restrict__ cnt, uint32_t *__restrict__ bits) {
    static_assert(kStage % kGroupTiles == 0 && kChunkTiles % kStage == 0, "stages hold whole groups");
    constexpr int kStageGroups = kStage / kGroupTiles;
    __shared__ __align__(16) float sc[kStage][kCen];
    __shared__ __align__(16) float sgc[kStageGroups][kCen];
    __shared__ float sr[kStage], sn[kStage], sgr[kStageGroups], sgn[kStageGroups];
    const int Q = blockIdx.x * kBoundThreads + threadIdx.x;
    const int chunk = blockIdx.y;
    const bool active = Q < qtiles;
    float c[kCen];
    const float4 *qc = reinterpret_cast<const float4 *>(qcen + (int64_t)(active ? Q : 0) * kCen);
#pragma unroll
    for (int u = 0; u < kCen / 4; ++u) {
        const float4 v = qc[u];
        c[4 * u] = v.x;
        c[4 * u + 1] = v.y;
        c[4 * u + 2] = v.z;
        c[4 * u + 3] = v.w;
    }
    const float rq = active ? qrad[Q] : 0.f, nq = active ? qn[Q] : 0.f, tq = active ? tau[Q] : INFINITY;
    // the query tile's window (already scanned by the first pass)
    const int tw = active ? Q / qpt : 0;
    const int wlo = max(0, tw - window), whi = min(dtiles, tw + window + 1);
    const int t0 = chunk * kChunkTiles, t1 = min(dtiles, t0 + kChunkTiles);
    uint32_t *wout = bits + ((int64_t)(active ? Q : 0) * nchunk + chunk) * kWords;
    int kept = 0;
    for (int s0 = t0, w = 0; s0 < t1; s0 += kStage, ++w) {
        const int ns = min(kStage, t1 - s0);
        const int ng = (ns + kGroupTiles - 1) / kGroupTiles;
        const int g0 = s0 / kGroupTiles;
        __syncthreads();
        for (int e = threadIdx.x; e < ns * kCen; e += blockDim.x) sc[e / kCen][e % kCen] = dcen[(int64_t)s0 * kCen + e];
        for (int e = threadIdx.x; e < ng * kCen; e += blockDim.x)
            sgc[e / kCen][e % kCen] = gcen[(int64_t)g0 * kCen + e];
        for (int e = threadIdx.x; e < ns; e += blockDim.x) {
            sr[e] = drad[s0 + e];
            sn[e] = dn[s0 + e];
        }
        for (int e = threadIdx.x; e < ng; e += blockDim.x) {
            sgr[e] = grad[g0 + e];
            sgn[e] = gn[g0 + e];
        }
        __syncthreads();
        uint32_t word = 0;
        for (int h = 0; h < ng; ++h) {
            if (!active || sphere_drop(c, sgc[h], sgr[h], sgn[h], rq, nq, tq, beta)) continue;
            const int e1 = min(ns, (h + 1) * kGroupTiles);
            for (int e = h * kGroupTiles; e < e1; ++e) {
                const int t = s0 + e;
                if (t >= wlo && t < whi) continue;
                if (!sphere_drop(c, sc[e], sr[e], sn[e], rq, nq, tq, beta)) word |= 1u << e;
            }
        }
        if (active) {
            wout[w] = word;
            kept += __popc(word);
        }
    }
    if (active) cnt[(int64_t)Q * nchunk + chunk] = kept;
}

// The kept tiles of (Q, chunk), ascending, from its bit words to
// tiles[off[Q * nchunk + chunk] ..] (entries past cap are dropped: the list
// pass then falls back to the full scan outside the window).
__global__ void __launch_bounds__(256)
fill_tiles_kernel(int qtiles, int dtiles, int nchunk, const uint32_t *__restrict__ bits,
                  const int64_t *__restrict__ off, int32_t *__restrict__ tiles, int64_t cap) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // Q * nchunk + chunk
    if (e >= (int64_t)qtiles * nchunk) return;
    const int chunk = (int)(e % nchunk);
    const uint32_t *win = bits + e * kWords;
    int64_t pos = off[e];
    const int t0 = chunk * kChunkTiles;
    const int nw = (int)ceil_div(min(dtiles - t0, kChunkTiles), kStage);
    for (int w = 0; w < nw; ++w) {
        uint32_t word = win[w];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            if (pos < cap) tiles[pos] = t0 + w * kStage + b;
            ++pos;
        }
    }
}

// tile_off[Q] = off[Q * nchunk] (the query tile's first chunk), tile_off[qtiles] = total.
__global__ void tile_offsets_kernel(int qtiles, int nchunk, const int64_t *__restrict__ off,
                                    int64_t *__restrict__ tile_off) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q <= qtiles) tile_off[Q] = off[(int64_t)Q * nchunk];
}

// Largest-first order of the list pass's items: query tiles by decreasing
// kept-tile count (counts bucketed by count >> shift into kOrderBins bins;
// order inside a bin is arbitrary).  A persistent launch that hands items out
// in this order ends on its smallest items, so its CTAs finish together.
// Item order does not change any result: every item owns its query rows.
constexpr int kOrderBins = 2048;

__global__ void __launch_bounds__(1024) item_order_kernel(const int64_t *__restrict__ tile_off, int items,
                                                          int shift, int32_t *__restrict__ order) {
    __shared__ int hist[kOrderBins];
    __shared__ int ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < kOrderBins; b += 1024) hist[b] = 0;
    __syncthreads();
    auto bin = [&](int i) {
        const int64_t c = (tile_off[i + 1] - tile_off[i]) >> shift;
        return kOrderBins - 1 - (int)(c < kOrderBins - 1 ? c : kOrderBins - 1);
    };
    for (int i = tid; i < items; i += 1024) atomicAdd(&hist[bin(i)], 1);
    __syncthreads();
    // exclusive scan, two bins per thread
    const int a0 = hist[2 * tid], a1 = hist[2 * tid + 1];
    int x = a0 + a1;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const int ex = x - a0 - a1 + (warp > 0 ? ws[warp - 1] : 0);
    hist[2 * tid] = ex;
    hist[2 * tid + 1] = ex + a0;
    __syncthreads();
    for (int i = tid; i < items; i += 1024) order[atomicAdd(&hist[bin(i)], 1)] = i;
}

// ---- batched search: items (query tile qt, sample t), item index t * T + qt

// Sample t's database tiles dtile_off[t] .. dtile_off[t + 1], staged kStage at
// a time; thread per query tile.  FN(local tile index, centre distance^2,
// radius, max norm) is called for every tile of t.
template <class FN>
__device__ __forceinline__ void for_sample_tiles(int t, const int32_t *__restrict__ dtile_off,
                                                 const float *__restrict__ dcen, const float *__restrict__ drad,
                                                 const float *__restrict__ dn, bool active, const float (&c)[kCen],
                                                 float (*sc)[kCen], float *sr, float *sn, FN fn) {
    const int g0 = dtile_off[t], g1 = dtile_off[t + 1];
    for (int s0 = g0; s0 < g1; s0 += kStage) {
        const int ns = min(kStage, g1 - s0);
        __syncthreads();
        for (int e = threadIdx.x; e < ns * kCen; e += blockDim.x) sc[e / kCen][e % kCen] = dcen[(int64_t)s0 * kCen + e];
        for (int e = threadIdx.x; e < ns; e += blockDim.x) {
            sr[e] = drad[s0 + e];
            sn[e] = dn[s0 + e];
        }
        __syncthreads();
        if (!active) continue;
        for (int e = 0; e < ns; ++e) {
            const float4 *dc = reinterpret_cast<const float4 *>(sc[e]);
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int u = 0; u < kCen / 4; u += 2) {
                const float4 x = dc[u], y = dc[u + 1];
                float f;
                f = c[4 * u] - x.x; a0 = fmaf(f, f, a0);
                f = c[4 * u + 1] - x.y; a0 = fmaf(f, f, a0);
                f = c[4 * u + 2] - x.z; a0 = fmaf(f, f, a0);
                f = c[4 * u + 3] - x.w; a0 = fmaf(f, f, a0);
                f = c[4 * u + 4] - y.x; a1 = fmaf(f, f, a1);
                f = c[4 * u + 5] - y.y; a1 = fmaf(f, f, a1);
                f = c[4 * u + 6] - y.z; a1 = fmaf(f, f, a1);
                f = c[4 * u + 7] - y.w; a1 = fmaf(f, f, a1);
            }
            fn(s0 + e - g0, a0 + a1, sr[e], sn[e]);
        }
    }
}

__device__ __forceinline__ void load_centre(const float *__restrict__ cen, int g, bool active, float (&c)[kCen]) {
    const float4 *qc = reinterpret_cast<const float4 *>(cen + (int64_t)(active ? g : 0) * kCen);
#pragma unroll
    for (int u = 0; u < kCen / 4; ++u) {
        const float4 v = qc[u];
        c[4 * u] = v.x;
        c[4 * u + 1] = v.y;
        c[4 * u + 2] = v.z;
        c[4 * u + 3] = v.w;
    }
}

// win[t * T + qt] = the tile of sample t whose centre is nearest query tile
// qt's (ties to the lower index).  Grid (query-tile blocks, samples).
__global__ void __launch_bounds__(kBoundThreads)
batched_nearest_kernel(int T, const int32_t *__restrict__ dtile_off, const float *__restrict__ qcen,
                       const float *__restrict__ dcen, const float *__restrict__ drad, const float *__restrict__ dn,
                       int32_t *__restrict__ win) {
    __shared__ __align__(16) float sc[kStage][kCen];
    __shared__ float sr[kStage], sn[kStage];
    const int qt = blockIdx.x * kBoundThreads + threadIdx.x, t = blockIdx.y;
    const bool active = qt < T;
    float c[kCen];
    load_centre(qcen, qt, active, c);
    float best = INFINITY;
    int bi = 0;
    for_sample_tiles(t, dtile_off, dcen, drad, dn, active, c, sc, sr, sn, [&](int m, float d2, float, float) {
        if (d2 < best) {
            best = d2;
            bi = m;
        }
    });
    if (active) win[(int64_t)t * T + qt] = bi;
}

// tau of item (qt, t) = max over the query tile's rows and parts of (saved
// threshold + |v_i|^2): the 16th key of a within list, the kShort-th of a
// cross list.  Warp per item.
__global__ void batched_tau_kernel(int64_t N, int T, int S, int parts, const int64_t *__restrict__ tile_row,
                                   const int64_t *__restrict__ tile_end, const int32_t *__restrict__ tile_samp,
                                   const float *__restrict__ st_w, const float *__restrict__ st_x,
                                   const float *__restrict__ row_norm, float *__restrict__ tau) {
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item >= (int64_t)T * S) return;
    const int t = (int)(item / T), qt = (int)(item - (int64_t)t * T);
    const bool within = tile_samp[qt] == t;
    float m = -INFINITY;
    for (int64_t q = tile_row[qt] + lane; q < tile_end[qt]; q += 32) {
        for (int p = 0; p < parts; ++p) {
            const float key = within ? st_w[((int64_t)p * N + q) * kBatchedList + kBatchedList - 1]
                                     : st_x[((q * S + t) * parts + p) * kBatchedShort + kBatchedShort - 1];
            m = fmaxf(m, key + row_norm[q]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) tau[item] = m;
}

// Kept tiles of item (qt, t): every tile of sample t outside the window
// [win - window, win + window] that the sphere bound cannot drop.  FILL =
// false: count into cnt[item]; FILL = true: write them, ascending, from
// off[item].  Grid (query-tile blocks, samples).
template <bool FILL>
__global__ void __launch_bounds__(kBoundThreads)
batched_prune_kernel(int T, int window, float beta, const int32_t *__restrict__ dtile_off,
                     const float *__restrict__ qcen, const float *__restrict__ qrad, const float *__restrict__ qn,
                     const float *__restrict__ tau, const int32_t *__restrict__ win, const float *__restrict__ dcen,
                     const float *__restrict__ drad, const float *__restrict__ dn, int32_t *__restrict__ cnt,
                     const int64_t *__restrict__ off, int32_t *__restrict__ tiles, int64_t cap) {
    __shared__ __align__(16) float sc[kStage][kCen];
    __shared__ float sr[kStage], sn[kStage];
    const int qt = blockIdx.x * kBoundThreads + threadIdx.x, t = blockIdx.y;
    const bool active = qt < T;
    const int64_t item = (int64_t)t * T + (active ? qt : 0);
    float c[kCen];
    load_centre(qcen, qt, active, c);
    const float rq = active ? qrad[qt] : 0.f, nq = active ? qn[qt] : 0.f, tq = active ? tau[item] : INFINITY;
    const int w = active ? win[item] : 0;
    int kept = 0;
    int64_t pos = (FILL && active) ? off[item] : 0;
    for_sample_tiles(t, dtile_off, dcen, drad, dn, active, c, sc, sr, sn, [&](int m, float d2, float rt, float nt) {
        if (m >= w - window && m <= w + window) return;
        const float gap = sqrtf(d2) - rq - rt;
        const float margin = 0x1p-11f * (nq + nt);
        const bool drop = gap > 0.f && gap * gap - beta * nt - margin > tq;
        if (!drop) {
            if (FILL && pos < cap) tiles[pos] = m;
            ++pos;
            ++kept;
        }
    });
    if (!FILL && active) cnt[item] = kept;
}

}  // namespace

PruneShape prune_shape(int64_t n, int BM, int BN) {
    PruneShape s;
    s.qtiles = (int)ceil_div(n, BM);
    s.dtiles = (int)ceil_div(n, BN);
    s.nchunk = (int)ceil_div(s.dtiles, kChunkTiles);
    const int64_t all = (int64_t)s.qtiles * s.dtiles;
    s.cap = std::min<int64_t>(all, kPruneListCap);
    return s;
}

// Layout of the pruning scratch (shared by the launcher and prune_outputs).
struct PruneLayout {
    float *row_norm, *qcen, *qrad, *qn, *dcen, *drad, *dn, *gcen, *grad, *gn, *tau;
    int32_t *cnt;
    uint32_t *bits;
    int64_t *off, *ssum;
    PruneOut out;
};

PruneLayout prune_layout(void *scratch, int64_t n, const PruneShape &s, size_t *bytes = nullptr) {
    Carve cv(scratch);
    PruneLayout L;
    L.row_norm = cv.take<float>((size_t)n);
    L.qcen = cv.take<float>((size_t)s.qtiles * kCen);
    L.qrad = cv.take<float>((size_t)s.qtiles);
    L.qn = cv.take<float>((size_t)s.qtiles);
    L.dcen = cv.take<float>((size_t)s.dtiles * kCen);
    L.drad = cv.take<float>((size_t)s.dtiles);
    L.dn = cv.take<float>((size_t)s.dtiles);
    const size_t ngroups = (size_t)ceil_div(s.dtiles, kGroupTiles);
    L.gcen = cv.take<float>(ngroups * kCen);
    L.grad = cv.take<float>(ngroups);
    L.gn = cv.take<float>(ngroups);
    L.tau = cv.take<float>((size_t)s.qtiles);
    const size_t ncnt = (size_t)s.qtiles * s.nchunk;
    L.cnt = cv.take<int32_t>(ncnt);
    L.bits = cv.take<uint32_t>(ncnt * kWords);
    L.off = cv.take<int64_t>(ncnt + 1);
    L.ssum = cv.take<int64_t>(seg_scan::kMaxSegs);
    L.out.tile_off = cv.take<int64_t>((size_t)s.qtiles + 1);
    L.out.tiles = cv.take<int32_t>((size_t)s.cap);
    L.out.order = cv.take<int32_t>((size_t)s.qtiles);
    L.out.overflow = cv.take<int32_t>(1);
    L.out.counter = cv.take<int32_t>(1);
    if (bytes) *bytes = cv.used;
    return L;
}

PruneOut prune_outputs(void *scratch, int64_t n, int BM, int BN) {
    return prune_layout(scratch, n, prune_shape(n, BM, BN)).out;
}

size_t prune_scratch_bytes(int64_t n, int BM, int BN) {
    size_t bytes = 0;
    prune_layout(nullptr, n, prune_shape(n, BM, BN), &bytes);
    return bytes;
}

cudaError_t launch_prune_bounds(const void *Qb, int64_t n, int d, int metric, int BM, int BN, int window,
                                const float *st_key, int EG, int KCP, void *scratch, PruneOut *out,
                                cudaStream_t st) {
    const PruneShape s = prune_shape(n, BM, BN);
    if (BN % BM != 0) return cudaErrorInvalidValue;
    const PruneLayout PL = prune_layout(scratch, n, s);
    float *row_norm = PL.row_norm, *qcen = PL.qcen, *qrad = PL.qrad, *qn = PL.qn;
    float *dcen = PL.dcen, *drad = PL.drad, *dn = PL.dn, *tau = PL.tau;
    int32_t *cnt = PL.cnt;
    int64_t *off = PL.off;
    *out = PL.out;
    const size_t ncnt = (size_t)s.qtiles * s.nchunk;
    const int W = 64 * tc_kb(d, metric);
    const int dv = metric == RSC_COSINE ? d + 1 : d;
    const float beta = metric == RSC_COSINE ? 1.f : 0.f;
    const uint16_t *q16 = static_cast<const uint16_t *>(Qb);
    tile_sphere_kernel<<<(unsigned)ceil_div((int64_t)s.qtiles * 32, 256), 256, 0, st>>>(
        q16, n, W, dv, BM, s.qtiles, nullptr, nullptr, qcen, qrad, qn, row_norm);
    tile_sphere_kernel<<<(unsigned)ceil_div((int64_t)s.dtiles * 32, 256), 256, 0, st>>>(
        q16, n, W, dv, BN, s.dtiles, nullptr, nullptr, dcen, drad, dn, nullptr);
    tile_tau_kernel<<<(unsigned)ceil_div((int64_t)s.qtiles * 32, 256), 256, 0, st>>>(st_key, n, EG, KCP, row_norm,
                                                                                     s.qtiles, BM, tau);
    const int ngroups = (int)ceil_div(s.dtiles, kGroupTiles);
    group_sphere_kernel<<<(unsigned)ceil_div((int64_t)ngroups * 32, 256), 256, 0, st>>>(
        dcen, drad, dn, s.dtiles, ngroups, PL.gcen, PL.grad, PL.gn);
    const dim3 grid((unsigned)ceil_div(s.qtiles, kBoundThreads), (unsigned)s.nchunk);
    const int qpt = BN / BM;
    prune_tiles_kernel<<<grid, kBoundThreads, 0, st>>>(s.qtiles, s.dtiles, s.nchunk, qpt, window, beta, qcen, qrad,
                                                       qn, tau, dcen, drad, dn, PL.gcen, PL.grad, PL.gn, cnt, PL.bits);
    cudaError_t e = seg_scan::launch(cnt, (int64_t)ncnt, off, PL.ssum, st, s.cap, out->overflow);
    if (e != cudaSuccess) return e;
    fill_tiles_kernel<<<(unsigned)ceil_div((int64_t)ncnt, 256), 256, 0, st>>>(s.qtiles, s.dtiles, s.nchunk, PL.bits,
                                                                             off, out->tiles, s.cap);
    tile_offsets_kernel<<<(unsigned)ceil_div(s.qtiles + 1, 256), 256, 0, st>>>(s.qtiles, s.nchunk, off,
                                                                               out->tile_off);
    int shift = 0;
    while ((s.dtiles >> shift) >= kOrderBins) ++shift;
    item_order_kernel<<<1, 1024, 0, st>>>(out->tile_off, s.qtiles, shift, out->order);
    return cudaGetLastError();
}


// ---- batched bounds: scratch layout and launchers

namespace {

struct BatchedPruneLayout {
    float *row_norm, *qcen, *qrad, *qn, *dcen, *drad, *dn, *tau;
    int32_t *cnt;
    int64_t *ssum;
    BatchedPruneOut out;
};

BatchedPruneLayout batched_prune_layout(void *scratch, int64_t N, int64_t T, int S, int64_t DT, size_t *bytes) {
    Carve cv(scratch);
    BatchedPruneLayout L;
    const size_t items = (size_t)T * S;
    L.row_norm = cv.take<float>((size_t)N);
    L.qcen = cv.take<float>((size_t)T * kCen);
    L.qrad = cv.take<float>((size_t)T);
    L.qn = cv.take<float>((size_t)T);
    L.dcen = cv.take<float>((size_t)DT * kCen);
    L.drad = cv.take<float>((size_t)DT);
    L.dn = cv.take<float>((size_t)DT);
    L.tau = cv.take<float>(items);
    L.cnt = cv.take<int32_t>(items);
    L.ssum = cv.take<int64_t>(seg_scan::kMaxSegs);
    L.out.win = cv.take<int32_t>(items);
    L.out.tile_off = cv.take<int64_t>(items + 1);
    L.out.tiles = cv.take<int32_t>((size_t)std::min<int64_t>((int64_t)items * std::max<int64_t>(DT / S, 1),
                                                             kPruneListCap));
    L.out.overflow = cv.take<int32_t>(1);
    if (bytes) *bytes = cv.used;
    return L;
}

int64_t batched_prune_cap(int64_t T, int S, int64_t DT) {
    return std::min<int64_t>(T * S * std::max<int64_t>(DT / S, 1), kPruneListCap);
}

}  // namespace

size_t batched_prune_scratch_bytes(int64_t N, int64_t T, int S, int64_t DT) {
    size_t bytes = 0;
    batched_prune_layout(nullptr, N, T, S, DT, &bytes);
    return bytes;
}

BatchedPruneOut batched_prune_outputs(void *scratch, int64_t N, int64_t T, int S, int64_t DT) {
    return batched_prune_layout(scratch, N, T, S, DT, nullptr).out;
}

cudaError_t launch_batched_prune_window(const void *Qb, int64_t N, int d, int metric, const void *tables_dev, int64_t T,
                                        int S, int64_t DT, void *scratch, cudaStream_t st) {
    const BatchedPruneLayout L = batched_prune_layout(scratch, N, T, S, DT, nullptr);
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    const int W = 64 * tc_kb(d, metric);
    const int dv = metric == RSC_COSINE ? d + 1 : d;
    const uint16_t *q16 = static_cast<const uint16_t *>(Qb);
    tile_sphere_kernel<<<(unsigned)ceil_div(T * 32, 256), 256, 0, st>>>(q16, N, W, dv, 0, (int)T, b.tile_row, b.tile_end,
                                                                       L.qcen, L.qrad, L.qn, L.row_norm);
    tile_sphere_kernel<<<(unsigned)ceil_div(DT * 32, 256), 256, 0, st>>>(q16, N, W, dv, 0, (int)DT, b.dtile_start,
                                                                        b.dtile_end, L.dcen, L.drad, L.dn, nullptr);
    const dim3 grid((unsigned)ceil_div(T, kBoundThreads), (unsigned)S);
    batched_nearest_kernel<<<grid, kBoundThreads, 0, st>>>((int)T, b.dtile_off, L.qcen, L.dcen, L.drad, L.dn,
                                                           L.out.win);
    return cudaGetLastError();
}

cudaError_t launch_batched_prune_bounds(int64_t N, int d, int metric, const void *tables_dev, int64_t T, int S,
                                        int64_t DT, int window, int parts, const float *st_w, const float *st_x,
                                        void *scratch, cudaStream_t st) {
    (void)d;
    const BatchedPruneLayout L = batched_prune_layout(scratch, N, T, S, DT, nullptr);
    const BatchedTables b = batched_tables(const_cast<void *>(tables_dev), T, S, DT);
    const int64_t items = T * S;
    const float beta = metric == RSC_COSINE ? 1.f : 0.f;
    const int64_t cap = batched_prune_cap(T, S, DT);
    batched_tau_kernel<<<(unsigned)ceil_div(items * 32, 256), 256, 0, st>>>(N, (int)T, S, parts, b.tile_row, b.tile_end,
                                                                           b.tile_samp, st_w, st_x, L.row_norm, L.tau);
    const dim3 grid((unsigned)ceil_div(T, kBoundThreads), (unsigned)S);
    batched_prune_kernel<false><<<grid, kBoundThreads, 0, st>>>((int)T, window, beta, b.dtile_off, L.qcen, L.qrad,
                                                                L.qn, L.tau, L.out.win, L.dcen, L.drad, L.dn, L.cnt,
                                                                nullptr, nullptr, cap);
    cudaError_t e = seg_scan::launch(L.cnt, items, L.out.tile_off, L.ssum, st, cap, L.out.overflow);
    if (e != cudaSuccess) return e;
    batched_prune_kernel<true><<<grid, kBoundThreads, 0, st>>>((int)T, window, beta, b.dtile_off, L.qcen, L.qrad,
                                                               L.qn, L.tau, L.out.win, L.dcen, L.drad, L.dn, nullptr,
                                                               L.out.tile_off, L.out.tiles, cap);
    return cudaGetLastError();
}

}  // namespace rsc
