// Leiden communities on the GPU: the clustering the paper runs on the stored
// neighbourhood graph (Methods, "Dimensionality reduction and graph
// analysis"), by the Leiden method (Traag, Waltman & van Eck 2019) with the
// modularity quality function and a resolution gamma.
//
// Every vertex of a round decides on the state the round began with, so a
// round is one launch over all vertices:
//   move     warp per vertex: the weights to each neighbouring community are
//            summed exactly and in no particular order: for rows of up to 32
//            entries in registers (lanes with equal labels found by
//            match.any, their weights added by redux.sync in 16-bit pieces),
//            for longer rows in an open-addressing table (64-bit atomic adds;
//            the warp's own table in shared memory up to 128 entries, the
//            vertex's table in global memory beyond; read back and cleared);
//            the warp picks
//            the community with the largest gain (128-bit integer gains, ties
//            to the smaller label);
//            moves alternate direction between rounds (even: to a smaller
//            label, odd: to a larger one);
//   refine   inside each community, vertices that are still alone and well
//            connected join the well-connected subcommunity of a neighbour
//            with the largest non-negative gain; a vertex someone picked stays;
//   aggregate one node per subcommunity (numbered by smallest member), the
//            node-to-node weights summed in per-node tables.
// Weights are fixed point (w * 2^32 rounded to a 64-bit integer), so every
// decision is exact and the partition is the same on every run; the host
// drives the rounds and levels (each round ends with a read of its move
// count).  rsc.h states the definition in full.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace rsc {

namespace ldn {

typedef __int128 i128;
typedef unsigned long long u64;

constexpr int kWarps = 8;   // warps per block of the per-vertex kernels
constexpr int kBlock = kWarps * 32;
constexpr int kCounters = 64;   // spread counters (moves, community counts)
constexpr int32_t kNone = INT32_MAX;
constexpr int kSmemSlots = 256;   // per-warp shared-memory table: rows of up to 128 entries

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Table length of a row of deg entries: a power of two >= 2 deg, at least 2.
__host__ __device__ __forceinline__ int64_t table_len(int64_t deg) {
    int64_t s = 2;
    while (s < 2 * deg) s <<= 1;
    return s;
}

// Adds w to key c's sum in the table [key, sum] of length len (a power of
// two with a free slot for every key ever inserted).
__device__ __forceinline__ void table_add(int32_t *key, u64 *sum, int64_t len, int32_t c, int64_t w) {
    int64_t s = (int64_t)(mix32((uint32_t)c) & (uint32_t)(len - 1));
    for (int64_t probe = 0; probe < len; ++probe) {
        const int32_t old = atomicCAS(key + s, -1, c);
        if (old == -1 || old == c) {
            atomicAdd(sum + s, (u64)w);
            return;
        }
        s = (s + 1) & (len - 1);
    }
}

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o) {
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    const uint64_t l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    return (i128)(((unsigned __int128)h2 << 64) | l2);
}

// Warp-wide best (largest gain, then smallest label); c == kNone: no candidate.
__device__ __forceinline__ void warp_best(i128 &g, int32_t &c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const i128 og = shfl_xor_i128(g, o);
        const int32_t oc = __shfl_xor_sync(0xffffffffu, c, o);
        if (oc != kNone && (c == kNone || og > g || (og == g && oc < c))) {
            g = og;
            c = oc;
        }
    }
}

// Rows of at most 32 entries, without tables: lane l holds entry l's label c
// (kNone when the entry is skipped) and weight w.  Lanes with equal labels
// find each other (match.any) and add their weights exactly in four 16-bit
// pieces (redux.sync.add over the lanes of the label); the label's first lane
// is its leader.  Returns the label's total weight.
__device__ __forceinline__ int64_t label_sum(int32_t c, int64_t w, bool &leader) {
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const uint64_t u = (uint64_t)w;
    const uint64_t p0 = __reduce_add_sync(peers, (unsigned)(u & 0xFFFF));
    const uint64_t p1 = __reduce_add_sync(peers, (unsigned)((u >> 16) & 0xFFFF));
    const uint64_t p2 = __reduce_add_sync(peers, (unsigned)((u >> 32) & 0xFFFF));
    const uint64_t p3 = __reduce_add_sync(peers, (unsigned)(u >> 48));
    leader = c != kNone && (int)(__ffs(peers) - 1) == (int)(threadIdx.x & 31);
    return (int64_t)(p0 + (p1 << 16) + (p2 << 32) + (p3 << 48));
}

__global__ void weights_kernel(const float *__restrict__ data, int64_t nnz, int64_t *__restrict__ wt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) wt[e] = __double2ll_rn((double)data[e] * 4294967296.0);
}

__global__ void check_graph_kernel(const int64_t *__restrict__ ip, const int32_t *__restrict__ col, int64_t n,
                                   int64_t nnz, unsigned int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (ip[i + 1] < ip[i] || ip[i] < 0 || ip[i + 1] > nnz)) record_status(status, RSC_ERR_INVALID_ARG);
    if (i < nnz && (col[i] < 0 || (int64_t)col[i] >= n)) record_status(status, RSC_ERR_INVALID_ARG);
}

__global__ void fill_kernel(int32_t *__restrict__ a, int64_t n, int32_t v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void iota_kernel(int32_t *__restrict__ a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

// Starting labels: the caller's partition (checked) or each vertex alone.
__global__ void init_comm_kernel(const int32_t *__restrict__ init, int64_t n, int32_t *__restrict__ comm,
                                 unsigned int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = init ? init[i] : (int32_t)i;
    if (c < 0 || (int64_t)c >= n) {
        record_status(status, RSC_ERR_INVALID_ARG);
        c = (int32_t)i;
    }
    comm[i] = c;
}

// Warp per vertex: strength k_v (the row sum), 2m, and the vertex table length.
__global__ void __launch_bounds__(kBlock)
strength_kernel(int64_t nv, const int64_t *__restrict__ ip, const int64_t *__restrict__ wt, int64_t *__restrict__ k,
                u64 *__restrict__ m2, int64_t *__restrict__ tlen) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= nv) return;
    int64_t s = 0;
    for (int64_t e = ip[v] + lane; e < ip[v + 1]; e += 32) s += wt[e];
    s = warp_sum(s);
    if (lane == 0) {
        k[v] = s;
        tlen[v] = table_len(ip[v + 1] - ip[v]);
        if (s) atomicAdd(m2 + (blockIdx.x & (kCounters - 1)), (u64)s);
    }
}

__global__ void tot_kernel(int64_t nv, const int32_t *__restrict__ lab, const int64_t *__restrict__ k,
                           u64 *__restrict__ tot) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv && k[v]) atomicAdd(tot + lab[v], (u64)k[v]);
}

// Relabel by smallest member: pass 1 takes the minima, pass 2 writes them.
__global__ void min_member_kernel(int64_t nv, const int32_t *__restrict__ lab, int32_t *__restrict__ minm) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) atomicMin(minm + lab[v], (int32_t)v);
}

__global__ void relabel_kernel(int64_t nv, int32_t *__restrict__ lab, const int32_t *__restrict__ minm) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) lab[v] = minm[lab[v]];
}

// Counts labels equal to their own index (communities after relabelling).
__global__ void count_self_kernel(int64_t nv, const int32_t *__restrict__ lab, u64 *__restrict__ cnt) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool self = v < nv && lab[v] == (int32_t)v;
    const unsigned b = __ballot_sync(0xffffffffu, self);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(cnt + (blockIdx.x & (kCounters - 1)), (u64)__popc(b));
}

// ---------------------------------------------------------------- moving

__global__ void __launch_bounds__(kBlock, 5)
move_kernel(int64_t nv, const int64_t *__restrict__ ip, const int32_t *__restrict__ col,
            const int64_t *__restrict__ wt, const int64_t *__restrict__ k, const u64 *__restrict__ tot,
            const int32_t *__restrict__ comm, int32_t *__restrict__ next, int64_t m2, int64_t G, int parity,
            const int64_t *__restrict__ toff, int32_t *__restrict__ hkey, u64 *__restrict__ hsum,
            u64 *__restrict__ moves) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= nv) return;   // warp-uniform
    const int32_t a = comm[v];
    const int64_t kv = k[v];
    const int64_t e0 = ip[v], e1 = ip[v + 1];
    int64_t sa = 0;
    i128 gb = 0;
    int32_t best = kNone;
    if (e1 - e0 <= 32) {   // warp-uniform: sums in registers
        int32_t c = kNone;
        int64_t w = 0;
        if (e0 + lane < e1) {
            const int32_t u = col[e0 + lane];
            w = wt[e0 + lane];
            if (u != v && w != 0) c = comm[u];
        }
        bool leader;
        const int64_t sc = label_sum(c, w, leader);
        if (leader) {
            if (c == a) {
                sa = sc;
            } else {
                gb = (i128)sc * m2 * 65536 - (i128)G * kv * (int64_t)tot[c];
                best = c;
            }
        }
    }
    // longer rows: a table in shared memory (up to 128 entries) or the
    // vertex's own table in global memory
    __shared__ int32_t s_key[kWarps][kSmemSlots];
    __shared__ u64 s_sum[kWarps][kSmemSlots];
    const int64_t deg = e1 - e0;
    const bool in_smem = deg > 32 && deg <= kSmemSlots / 2;
    int64_t len = 0;
    int32_t *key;
    u64 *sum;
    if (in_smem) {
        len = table_len(deg);
        key = s_key[(threadIdx.x >> 5)];
        sum = s_sum[(threadIdx.x >> 5)];
        for (int64_t s = lane; s < len; s += 32) {
            key[s] = -1;
            sum[s] = 0;
        }
        __syncwarp();
    } else {
        const int64_t T = toff[v];
        len = deg <= 32 ? 0 : toff[v + 1] - T;
        key = hkey + T;
        sum = hsum + T;
    }
    for (int64_t e = e0 + lane; e < e1 && len; e += 32) {
        const int32_t u = col[e];
        const int64_t w = wt[e];
        if (u != v && w != 0) table_add(key, sum, len, comm[u], w);
    }
    __syncwarp();
    for (int64_t s = lane; s < len; s += 32) {
        const int32_t c = in_smem ? key[s] : __ldcg(key + s);
        if (c < 0) continue;
        const int64_t sc = (int64_t)(in_smem ? sum[s] : __ldcg(sum + s));
        key[s] = -1;
        sum[s] = 0;
        if (c == a) {
            sa = sc;
            continue;
        }
        const i128 g = (i128)sc * m2 * 65536 - (i128)G * kv * (int64_t)tot[c];
        if (best == kNone || g > gb || (g == gb && c < best)) {
            gb = g;
            best = c;
        }
    }
    sa = warp_sum(sa);
    warp_best(gb, best);
    if (lane == 0) {
        const i128 ga = (i128)sa * m2 * 65536 - (i128)G * kv * ((int64_t)tot[a] - kv);
        int32_t nb = a;
        if (best != kNone && gb > ga && (parity == 0 ? best < a : best > a)) nb = best;
        next[v] = nb;
        if (nb != a) atomicAdd(moves + (blockIdx.x & (kCounters - 1)), 1ull);
    }
}

// ------------------------------------------------------------ refinement

// Warp per vertex: weight to the other vertices of its own community (mode 0:
// by comm, into wC) or of its own subcommunity (mode 1: by ref, into the
// subcommunity statistics).
__global__ void __launch_bounds__(kBlock)
inner_kernel(int64_t nv, const int64_t *__restrict__ ip, const int32_t *__restrict__ col,
             const int64_t *__restrict__ wt, const int64_t *__restrict__ k, const int32_t *__restrict__ lab, int mode,
             int64_t *__restrict__ wC, u64 *__restrict__ rtot, u64 *__restrict__ ext, int32_t *__restrict__ size) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= nv) return;
    const int32_t l = lab[v];
    int64_t s = 0;
    for (int64_t e = ip[v] + lane; e < ip[v + 1]; e += 32) {
        const int32_t u = col[e];
        if (u != v && lab[u] == l) s += wt[e];
    }
    s = warp_sum(s);
    if (lane == 0) {
        if (mode == 0) {
            wC[v] = s;
        } else {
            atomicAdd(rtot + l, (u64)k[v]);
            atomicAdd(size + l, 1);
            atomicAdd(ext + l, (u64)(wC[v] - s));
        }
    }
}

__global__ void __launch_bounds__(kBlock, 5)
pick_kernel(int64_t nv, const int64_t *__restrict__ ip, const int32_t *__restrict__ col,
            const int64_t *__restrict__ wt, const int64_t *__restrict__ k, const u64 *__restrict__ tot,
            const int32_t *__restrict__ comm, const int32_t *__restrict__ ref, const int64_t *__restrict__ wC,
            const u64 *__restrict__ rtot, const u64 *__restrict__ ext, const int32_t *__restrict__ size,
            int64_t m2, int64_t G, const int64_t *__restrict__ toff, int32_t *__restrict__ hkey,
            u64 *__restrict__ hsum, int32_t *__restrict__ target, int32_t *__restrict__ picked) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= nv) return;
    const int32_t C = comm[v], own = ref[v];
    const int64_t kv = k[v], totC = (int64_t)tot[C];
    // only vertices still alone and well connected to their community move
    if (size[own] != 1 || (i128)wC[v] * m2 * 65536 < (i128)G * kv * (totC - kv)) {
        if (lane == 0) target[v] = -1;
        return;
    }
    const int64_t e0 = ip[v], e1 = ip[v + 1];
    i128 gb = 0;
    int32_t best = kNone;
    if (e1 - e0 <= 32) {   // warp-uniform: sums in registers
        int32_t S = kNone;
        int64_t w = 0;
        if (e0 + lane < e1) {
            const int32_t u = col[e0 + lane];
            w = wt[e0 + lane];
            if (u != v && w != 0 && comm[u] == C) S = ref[u];
        }
        bool leader;
        const int64_t sS = label_sum(S, w, leader);
        if (leader && S != own) {
            const int64_t rS = (int64_t)rtot[S];
            if ((i128)(int64_t)ext[S] * m2 * 65536 >= (i128)G * rS * (totC - rS)) {
                const i128 g = (i128)sS * m2 * 65536 - (i128)G * kv * rS;
                if (g >= 0) {
                    gb = g;
                    best = S;
                }
            }
        }
    }
    __shared__ int32_t s_key[kWarps][kSmemSlots];
    __shared__ u64 s_sum[kWarps][kSmemSlots];
    const int64_t deg = e1 - e0;
    const bool in_smem = deg > 32 && deg <= kSmemSlots / 2;
    int64_t len = 0;
    int32_t *key;
    u64 *sum;
    if (in_smem) {
        len = table_len(deg);
        key = s_key[(threadIdx.x >> 5)];
        sum = s_sum[(threadIdx.x >> 5)];
        for (int64_t s = lane; s < len; s += 32) {
            key[s] = -1;
            sum[s] = 0;
        }
        __syncwarp();
    } else {
        const int64_t T = toff[v];
        len = deg <= 32 ? 0 : toff[v + 1] - T;
        key = hkey + T;
        sum = hsum + T;
    }
    for (int64_t e = e0 + lane; e < e1 && len; e += 32) {
        const int32_t u = col[e];
        const int64_t w = wt[e];
        if (u != v && w != 0 && comm[u] == C) table_add(key, sum, len, ref[u], w);
    }
    __syncwarp();
    for (int64_t s = lane; s < len; s += 32) {
        const int32_t S = in_smem ? key[s] : __ldcg(key + s);
        if (S < 0) continue;
        const int64_t sS = (int64_t)(in_smem ? sum[s] : __ldcg(sum + s));
        key[s] = -1;
        sum[s] = 0;
        if (S == own) continue;
        const int64_t rS = (int64_t)rtot[S];
        if ((i128)(int64_t)ext[S] * m2 * 65536 < (i128)G * rS * (totC - rS)) continue;
        const i128 g = (i128)sS * m2 * 65536 - (i128)G * kv * rS;
        if (g < 0) continue;
        if (best == kNone || g > gb || (g == gb && S < best)) {
            gb = g;
            best = S;
        }
    }
    warp_best(gb, best);
    if (lane == 0) {
        target[v] = best == kNone ? -1 : best;
        if (best != kNone) picked[best] = 1;
    }
}

__global__ void apply_kernel(int64_t nv, const int32_t *__restrict__ target, const int32_t *__restrict__ picked,
                             int32_t *__restrict__ ref, u64 *__restrict__ moves) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (v < nv) {
        const int32_t t = target[v];
        if (t >= 0 && !picked[ref[v]]) {
            ref[v] = t;
            mv = true;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, mv);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(moves + (blockIdx.x & (kCounters - 1)), (u64)__popc(b));
}

// ----------------------------------------------------------- aggregation

__global__ void head_flag_kernel(int64_t nv, const int32_t *__restrict__ ref, int32_t *__restrict__ flag) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) flag[v] = ref[v] == (int32_t)v;
}

// node[v] = index of v's subcommunity; the aggregate's communities; each
// node's entry count; the original vertices' nodes one level up.
__global__ void node_kernel(int64_t nv, const int32_t *__restrict__ ref, const int64_t *__restrict__ pos,
                            const int32_t *__restrict__ comm, const int64_t *__restrict__ ip, int32_t *__restrict__ node,
                            int32_t *__restrict__ ncomm, u64 *__restrict__ ndeg) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int32_t c = (int32_t)pos[ref[v]];
    node[v] = c;
    ncomm[c] = (int32_t)pos[ref[comm[v]]];   // comm[v] is its community's smallest member
    atomicAdd(ndeg + c, (u64)(ip[v + 1] - ip[v]));
}

__global__ void top_kernel(int64_t n, const int32_t *__restrict__ node, int32_t *__restrict__ top) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) top[i] = node[top[i]];
}

__global__ void node_tlen_kernel(int64_t K, const u64 *__restrict__ ndeg, int64_t *__restrict__ tlen) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < K) tlen[c] = table_len((int64_t)ndeg[c]);
}

__global__ void __launch_bounds__(kBlock)
agg_insert_kernel(int64_t nv, const int64_t *__restrict__ ip, const int32_t *__restrict__ col,
                  const int64_t *__restrict__ wt, const int32_t *__restrict__ node, const int64_t *__restrict__ toff,
                  int32_t *__restrict__ hkey, u64 *__restrict__ hsum) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= nv) return;
    const int32_t c = node[v];
    const int64_t T = toff[c], len = toff[c + 1] - T;
    for (int64_t e = ip[v] + lane; e < ip[v + 1]; e += 32) {
        const int64_t w = wt[e];
        if (w != 0) table_add(hkey + T, hsum + T, len, node[col[e]], w);
    }
}

// Warp per node: mode 0 counts the used slots, mode 1 writes them (in slot
// order) to the aggregate's row and clears the table.
__global__ void __launch_bounds__(kBlock)
agg_row_kernel(int64_t K, const int64_t *__restrict__ toff, int32_t *__restrict__ hkey, u64 *__restrict__ hsum,
               int mode, int64_t *__restrict__ cnt, const int64_t *__restrict__ nip, int32_t *__restrict__ ncol,
               int64_t *__restrict__ nwt) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= K) return;
    const int64_t T = toff[c], len = toff[c + 1] - T;
    int64_t run = mode ? nip[c] : 0;
    for (int64_t s0 = 0; s0 < len; s0 += 32) {
        const int64_t s = s0 + lane;
        const int32_t t = s < len ? __ldcg(hkey + T + s) : -1;
        const unsigned b = __ballot_sync(0xffffffffu, t >= 0);
        if (mode && t >= 0) {
            const int64_t p = run + __popc(b & ((1u << lane) - 1u));
            ncol[p] = t;
            nwt[p] = (int64_t)__ldcg(hsum + T + s);
            hkey[T + s] = -1;
            hsum[T + s] = 0;
        }
        run += __popc(b);
    }
    if (!mode && lane == 0) cnt[c] = run;
}

// ------------------------------------------------------------- output

__global__ void member_kernel(int64_t n, const int32_t *__restrict__ comm, const int32_t *__restrict__ top,
                              int32_t *__restrict__ mem) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mem[i] = comm[top[i]];
}

// Numbering by first appearance: first[c] = smallest vertex of c; a vertex
// that is its label's first is flagged; the exclusive scan of the flags at
// first[c] is c's number.
__global__ void first_flag_kernel(int64_t n, const int32_t *__restrict__ mem, const int32_t *__restrict__ first,
                                  int32_t *__restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = first[mem[i]] == (int32_t)i;
}

__global__ void number_kernel(int64_t n, int32_t *__restrict__ mem, const int32_t *__restrict__ first,
                              const int64_t *__restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mem[i] = (int32_t)pos[first[mem[i]]];
}

// Per final community: weight inside (both directions) and total strength.
__global__ void __launch_bounds__(kBlock)
quality_kernel(int64_t n, const int64_t *__restrict__ ip, const int32_t *__restrict__ col,
               const int64_t *__restrict__ wt, const int32_t *__restrict__ mem, u64 *__restrict__ in_c,
               u64 *__restrict__ tot_c) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;
    const int32_t c = mem[v];
    int64_t a = 0, b = 0;
    for (int64_t e = ip[v] + lane; e < ip[v + 1]; e += 32) {
        a += wt[e];
        if (mem[col[e]] == c) b += wt[e];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        if (a) atomicAdd(tot_c + c, (u64)a);
        if (b) atomicAdd(in_c + c, (u64)b);
    }
}

}  // namespace ldn

namespace {

using ldn::u64;

struct LdLayout {
    unsigned int *status;
    u64 *cnt;                        // kCounters spread counters
    int64_t *ssum;                   // scan scratch
    int64_t *ip0, *wt0;              // level-0 graph (weights in fixed point)
    int32_t *col0;
    int64_t *ipA, *wtA, *ipB, *wtB;  // aggregated graphs
    int32_t *colA, *colB;
    int64_t *toff, *tlen;            // table offsets / lengths [n + 1]
    int32_t *hkey;
    u64 *hsum;
    int64_t *k, *wC, *pos;
    u64 *tot, *rtot, *ext, *ndeg;
    int32_t *comm, *next, *ref, *target, *picked, *size, *node, *top, *minm, *flag, *mem;
    int64_t hcap;
};

LdLayout carve_leiden(void *ws, int64_t n, int64_t nnz, size_t *bytes) {
    Carve cv(ws);
    LdLayout L;
    const size_t N = (size_t)n, E = (size_t)std::max<int64_t>(nnz, 1);
    L.status = cv.take<unsigned int>(kStatusBytes / sizeof(unsigned int));
    L.cnt = cv.take<u64>(ldn::kCounters);
    L.ssum = cv.take<int64_t>(seg_scan::kMaxSegs);
    L.ip0 = cv.take<int64_t>(N + 1);
    L.col0 = cv.take<int32_t>(E);
    L.wt0 = cv.take<int64_t>(E);
    L.ipA = cv.take<int64_t>(N + 1);
    L.colA = cv.take<int32_t>(E);
    L.wtA = cv.take<int64_t>(E);
    L.ipB = cv.take<int64_t>(N + 1);
    L.colB = cv.take<int32_t>(E);
    L.wtB = cv.take<int64_t>(E);
    L.toff = cv.take<int64_t>(N + 1);
    L.tlen = cv.take<int64_t>(N + 1);
    L.hcap = 4 * (int64_t)E + 2 * (int64_t)N + 64;
    L.hkey = cv.take<int32_t>((size_t)L.hcap);
    L.hsum = cv.take<u64>((size_t)L.hcap);
    L.k = cv.take<int64_t>(N);
    L.wC = cv.take<int64_t>(N);
    L.pos = cv.take<int64_t>(N + 1);
    L.tot = cv.take<u64>(N);
    L.rtot = cv.take<u64>(N);
    L.ext = cv.take<u64>(N);
    L.ndeg = cv.take<u64>(N);
    L.comm = cv.take<int32_t>(N);
    L.next = cv.take<int32_t>(N);
    L.ref = cv.take<int32_t>(N);
    L.target = cv.take<int32_t>(N);
    L.picked = cv.take<int32_t>(N);
    L.size = cv.take<int32_t>(N);
    L.node = cv.take<int32_t>(N);
    L.top = cv.take<int32_t>(N);
    L.minm = cv.take<int32_t>(N);
    L.flag = cv.take<int32_t>(N);
    L.mem = cv.take<int32_t>(N);
    if (bytes) *bytes = cv.used;
    return L;
}

// Sum of the spread counters (synchronises the stream), then clears them.
rsc_status read_counter(const LdLayout &L, cudaStream_t st, u64 *out) {
    u64 h[ldn::kCounters];
    RSC_CUDA_TRY(cudaMemcpyAsync(h, L.cnt, sizeof h, cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    u64 s = 0;
    for (int i = 0; i < ldn::kCounters; ++i) s += h[i];
    *out = s;
    RSC_CUDA_TRY(cudaMemsetAsync(L.cnt, 0, sizeof h, st));
    return RSC_OK;
}

inline unsigned blocks(int64_t threads, int per = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(threads, per)); }

// Relabel lab[0 .. nv) by smallest member.
rsc_status canon(const LdLayout &L, int64_t nv, int32_t *lab, cudaStream_t st) {
    ldn::fill_kernel<<<blocks(nv), 256, 0, st>>>(L.minm, nv, INT32_MAX);
    ldn::min_member_kernel<<<blocks(nv), 256, 0, st>>>(nv, lab, L.minm);
    ldn::relabel_kernel<<<blocks(nv), 256, 0, st>>>(nv, lab, L.minm);
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

rsc_status compute_tot(const LdLayout &L, int64_t nv, const int32_t *lab, u64 *tot, cudaStream_t st) {
    RSC_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(u64) * (size_t)nv, st));
    ldn::tot_kernel<<<blocks(nv), 256, 0, st>>>(nv, lab, L.k, tot);
    RSC_CUDA_TRY(cudaGetLastError());
    return RSC_OK;
}

struct LdParams {
    double gamma;
    int64_t G;
    int n_iter, max_levels, max_rounds;
};

rsc_status leiden_params(int64_t n, int64_t nnz, const rsc_leiden_opts *o, LdParams *p) {
    if (n < 1 || n >= (int64_t)INT32_MAX) return fail(RSC_ERR_INVALID_ARG, "n = %lld outside [1, 2^31)", (long long)n);
    if (nnz < 0 || nnz >= ((int64_t)1 << 40)) return fail(RSC_ERR_INVALID_ARG, "nnz = %lld out of range", (long long)nnz);
    const rsc_leiden_opts z{};
    const rsc_leiden_opts &q = o ? *o : z;
    const double gamma = q.resolution == 0.0 ? 1.0 : q.resolution;
    if (!(gamma > 0.0) || !(gamma < 32768.0)) return fail(RSC_ERR_INVALID_ARG, "resolution outside (0, 32768)");
    p->gamma = gamma;
    p->G = (int64_t)llrint(gamma * 65536.0);
    p->n_iter = q.n_iterations ? q.n_iterations : 2;
    p->max_levels = q.max_levels ? q.max_levels : 32;
    p->max_rounds = q.max_rounds ? q.max_rounds : 8;
    if (p->n_iter < 1 || p->n_iter > 1000 || p->max_levels < 1 || p->max_levels > 1000 || p->max_rounds < 1 ||
        p->max_rounds > 100000)
        return fail(RSC_ERR_INVALID_ARG, "n_iterations, max_levels or max_rounds out of range");
    return RSC_OK;
}

// Work of the last rsc_leiden call on this thread (rsc_leiden_last_stats).
struct LdStats {
    int64_t levels = 0, move_rounds = 0, refine_rounds = 0, entries = 0, vertices = 0, launches = 0;
};
thread_local LdStats g_last_stats;

// One level's table offsets from tlen [nv].
rsc_status table_offsets(const LdLayout &L, int64_t nv, cudaStream_t st) {
    RSC_CUDA_TRY(seg_scan::launch(L.tlen, nv, L.toff, L.ssum, st));
    return RSC_OK;
}

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" {

rsc_status rsc_leiden_last_stats(int64_t *stats) {
    if (!stats) return fail(RSC_ERR_INVALID_ARG, "stats is NULL");
    stats[0] = g_last_stats.levels;
    stats[1] = g_last_stats.move_rounds;
    stats[2] = g_last_stats.refine_rounds;
    stats[3] = g_last_stats.entries;
    stats[4] = g_last_stats.vertices;
    stats[5] = g_last_stats.launches;
    return RSC_OK;
}

rsc_status rsc_leiden_workspace_size(int64_t n, int64_t nnz, size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    LdParams p;
    rsc_status s = leiden_params(n, nnz, nullptr, &p);
    if (s != RSC_OK) return s;
    carve_leiden(nullptr, n, nnz, bytes);
    return RSC_OK;
}

rsc_status rsc_leiden(const int64_t *indptr, const int32_t *indices, const float *data, int64_t n, int64_t nnz,
                      const int32_t *init, int32_t *membership, int64_t *n_communities, double *modularity,
                      const rsc_leiden_opts *opts, void *workspace, size_t workspace_bytes) {
    RSC_TRACE("rsc_leiden");
    LdParams p;
    rsc_status s = leiden_params(n, nnz, opts, &p);
    if (s != RSC_OK) return s;
    if (!indptr || (nnz > 0 && (!indices || !data)) || !membership)
        return fail(RSC_ERR_INVALID_ARG, "indptr, indices, data or membership is NULL");
    size_t need = 0;
    carve_leiden(nullptr, n, nnz, &need);
    if (!workspace) return fail(RSC_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(RSC_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (workspace_bytes < need) return fail(RSC_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, need);
    LdLayout L = carve_leiden(workspace, n, nnz, nullptr);
    cudaStream_t st = static_cast<cudaStream_t>(opts ? opts->stream : nullptr);
    RSC_CUDA_TRY(cudaMemsetAsync(L.status, 0, kStatusBytes, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.cnt, 0, sizeof(u64) * ldn::kCounters, st));
    // level-0 graph: the caller's structure, fixed-point weights; checked
    RSC_CUDA_TRY(cudaMemcpyAsync(L.ip0, indptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, st));
    if (nnz > 0) {
        RSC_CUDA_TRY(cudaMemcpyAsync(L.col0, indices, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
        ldn::weights_kernel<<<blocks(nnz), 256, 0, st>>>(data, nnz, L.wt0);
    }
    ldn::check_graph_kernel<<<blocks(std::max(n, nnz)), 256, 0, st>>>(L.ip0, L.col0, n, nnz, L.status);
    ldn::init_comm_kernel<<<blocks(n), 256, 0, st>>>(init, n, L.mem, L.status);
    RSC_CUDA_TRY(cudaGetLastError());
    {
        unsigned int bad = 0;
        RSC_CUDA_TRY(cudaMemcpyAsync(&bad, L.status, sizeof bad, cudaMemcpyDeviceToHost, st));
        RSC_CUDA_TRY(cudaStreamSynchronize(st));
        if (bad) return fail(RSC_ERR_INVALID_ARG, "graph structure or starting labels out of range");
    }
    LdStats stats;
    g_last_stats = stats;
    stats.launches = (nnz > 0 ? 3 : 2);   // weights, checks, starting labels
    RSC_CUDA_TRY(cudaMemsetAsync(L.hkey, 0xFF, sizeof(int32_t) * (size_t)L.hcap, st));
    RSC_CUDA_TRY(cudaMemsetAsync(L.hsum, 0, sizeof(u64) * (size_t)L.hcap, st));
    for (int it = 0; it < p.n_iter; ++it) {
        const int64_t *ip = L.ip0;
        const int32_t *col = L.col0;
        const int64_t *wt = L.wt0;
        int64_t nv = n;
        bool useA = true;   // next aggregate goes to A, then B, alternately
        ldn::iota_kernel<<<blocks(n), 256, 0, st>>>(L.top, n);
        RSC_CUDA_TRY(cudaMemcpyAsync(L.comm, L.mem, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        if ((s = canon(L, n, L.comm, st)) != RSC_OK) return s;
        stats.launches += 4 + 1;   // ids, relabelling; the membership at the end of the run
        for (int level = 0; level < p.max_levels; ++level) {
            ++stats.levels;
            int64_t level_nnz = 0;
            RSC_CUDA_TRY(cudaMemcpyAsync(&level_nnz, ip + nv, sizeof level_nnz, cudaMemcpyDeviceToHost, st));
            // strengths, 2m, vertex tables
            const unsigned vb = blocks(nv * 32, ldn::kBlock);
            ldn::strength_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, wt, L.k, L.cnt, L.tlen);
            RSC_CUDA_TRY(cudaGetLastError());
            u64 m2u = 0;
            if ((s = read_counter(L, st, &m2u)) != RSC_OK) return s;
            const int64_t m2 = (int64_t)m2u;
            stats.launches += 1;
            if (m2 == 0) break;
            stats.launches += 2 + 5;   // table offsets; relabelling, totals and count after moving
            if ((s = table_offsets(L, nv, st)) != RSC_OK) return s;
            // 1. local moving
            int quiet = 0;
            for (int r = 0; r < p.max_rounds && quiet < 2; ++r) {
                if ((s = compute_tot(L, nv, L.comm, L.tot, st)) != RSC_OK) return s;
                ldn::move_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, col, wt, L.k, L.tot, L.comm, L.next, m2, p.G,
                                                             r % 2, L.toff, L.hkey, L.hsum, L.cnt);
                RSC_CUDA_TRY(cudaGetLastError());
                u64 moves = 0;
                if ((s = read_counter(L, st, &moves)) != RSC_OK) return s;
                ++stats.move_rounds;
                stats.launches += 2;
                stats.entries += level_nnz;
                stats.vertices += nv;
                std::swap(L.comm, L.next);
                quiet = moves ? 0 : quiet + 1;
            }
            if ((s = canon(L, nv, L.comm, st)) != RSC_OK) return s;
            if ((s = compute_tot(L, nv, L.comm, L.tot, st)) != RSC_OK) return s;
            ldn::count_self_kernel<<<blocks(nv), 256, 0, st>>>(nv, L.comm, L.cnt);
            u64 ncomm = 0;
            if ((s = read_counter(L, st, &ncomm)) != RSC_OK) return s;
            if ((int64_t)ncomm == nv) break;
            stats.launches += 2 + 3 + 3;   // refinement set-up; relabelling; head flags and their scan
            // 2. refinement
            ldn::inner_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, col, wt, L.k, L.comm, 0, L.wC, nullptr, nullptr,
                                                          nullptr);
            ldn::iota_kernel<<<blocks(nv), 256, 0, st>>>(L.ref, nv);
            for (int r = 0; r < p.max_rounds; ++r) {
                RSC_CUDA_TRY(cudaMemsetAsync(L.rtot, 0, sizeof(u64) * (size_t)nv, st));
                RSC_CUDA_TRY(cudaMemsetAsync(L.ext, 0, sizeof(u64) * (size_t)nv, st));
                RSC_CUDA_TRY(cudaMemsetAsync(L.size, 0, sizeof(int32_t) * (size_t)nv, st));
                RSC_CUDA_TRY(cudaMemsetAsync(L.picked, 0, sizeof(int32_t) * (size_t)nv, st));
                ldn::inner_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, col, wt, L.k, L.ref, 1, L.wC, L.rtot, L.ext,
                                                              L.size);
                ldn::pick_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, col, wt, L.k, L.tot, L.comm, L.ref, L.wC, L.rtot,
                                                             L.ext, L.size, m2, p.G, L.toff, L.hkey, L.hsum, L.target,
                                                             L.picked);
                ldn::apply_kernel<<<blocks(nv), 256, 0, st>>>(nv, L.target, L.picked, L.ref, L.cnt);
                RSC_CUDA_TRY(cudaGetLastError());
                u64 moves = 0;
                if ((s = read_counter(L, st, &moves)) != RSC_OK) return s;
                ++stats.refine_rounds;
                stats.launches += 3;
                stats.entries += 2 * level_nnz;   // the statistics pass and the picks
                stats.vertices += 2 * nv;
                if (!moves) break;
            }
            if ((s = canon(L, nv, L.ref, st)) != RSC_OK) return s;
            // 3. aggregation
            ldn::head_flag_kernel<<<blocks(nv), 256, 0, st>>>(nv, L.ref, L.flag);
            RSC_CUDA_TRY(seg_scan::launch(L.flag, nv, L.pos, L.ssum, st));
            int64_t K = 0;
            RSC_CUDA_TRY(cudaMemcpyAsync(&K, L.pos + nv, sizeof K, cudaMemcpyDeviceToHost, st));
            RSC_CUDA_TRY(cudaStreamSynchronize(st));
            if (K == nv) break;   // the refinement merged nothing
            stats.launches += 10;
            RSC_CUDA_TRY(cudaMemsetAsync(L.ndeg, 0, sizeof(u64) * (size_t)K, st));
            ldn::node_kernel<<<blocks(nv), 256, 0, st>>>(nv, L.ref, L.pos, L.comm, ip, L.node, L.next, L.ndeg);
            ldn::top_kernel<<<blocks(n), 256, 0, st>>>(n, L.node, L.top);
            ldn::node_tlen_kernel<<<blocks(K), 256, 0, st>>>(K, L.ndeg, L.tlen);
            RSC_CUDA_TRY(cudaGetLastError());
            if ((s = table_offsets(L, K, st)) != RSC_OK) return s;
            ldn::agg_insert_kernel<<<vb, ldn::kBlock, 0, st>>>(nv, ip, col, wt, L.node, L.toff, L.hkey, L.hsum);
            int64_t *nip = useA ? L.ipA : L.ipB;
            int32_t *ncol = useA ? L.colA : L.colB;
            int64_t *nwt = useA ? L.wtA : L.wtB;
            const unsigned kb = blocks(K * 32, ldn::kBlock);
            ldn::agg_row_kernel<<<kb, ldn::kBlock, 0, st>>>(K, L.toff, L.hkey, L.hsum, 0, L.tlen, nullptr, nullptr,
                                                            nullptr);
            RSC_CUDA_TRY(seg_scan::launch(L.tlen, K, nip, L.ssum, st));
            ldn::agg_row_kernel<<<kb, ldn::kBlock, 0, st>>>(K, L.toff, L.hkey, L.hsum, 1, nullptr, nip, ncol, nwt);
            RSC_CUDA_TRY(cudaGetLastError());
            // the aggregate's communities (written to next by node_kernel)
            RSC_CUDA_TRY(cudaMemcpyAsync(L.comm, L.next, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToDevice, st));
            ip = nip;
            col = ncol;
            wt = nwt;
            nv = K;
            useA = !useA;
        }
        ldn::member_kernel<<<blocks(n), 256, 0, st>>>(n, L.comm, L.top, L.mem);
        RSC_CUDA_TRY(cudaGetLastError());
    }
    // numbering by first appearance
    ldn::fill_kernel<<<blocks(n), 256, 0, st>>>(L.minm, n, INT32_MAX);
    ldn::min_member_kernel<<<blocks(n), 256, 0, st>>>(n, L.mem, L.minm);
    ldn::first_flag_kernel<<<blocks(n), 256, 0, st>>>(n, L.mem, L.minm, L.flag);
    RSC_CUDA_TRY(seg_scan::launch(L.flag, n, L.pos, L.ssum, st));
    ldn::number_kernel<<<blocks(n), 256, 0, st>>>(n, L.mem, L.minm, L.pos);
    RSC_CUDA_TRY(cudaMemcpyAsync(membership, L.mem, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    RSC_CUDA_TRY(cudaGetLastError());
    int64_t K = 0;
    RSC_CUDA_TRY(cudaMemcpyAsync(&K, L.pos + n, sizeof K, cudaMemcpyDeviceToHost, st));
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_communities) *n_communities = K;
    stats.launches += 6 + (modularity ? 1 : 0);
    g_last_stats = stats;
    if (modularity) {
        // per community inside weight and strength; summed on the host in
        // community order
        RSC_CUDA_TRY(cudaMemsetAsync(L.rtot, 0, sizeof(u64) * (size_t)K, st));
        RSC_CUDA_TRY(cudaMemsetAsync(L.tot, 0, sizeof(u64) * (size_t)K, st));
        ldn::quality_kernel<<<blocks(n * 32, ldn::kBlock), ldn::kBlock, 0, st>>>(n, L.ip0, L.col0, L.wt0, L.mem,
                                                                                 L.rtot, L.tot);
        RSC_CUDA_TRY(cudaGetLastError());
        std::vector<u64> in_c((size_t)K), tot_c((size_t)K);
        RSC_CUDA_TRY(cudaMemcpyAsync(in_c.data(), L.rtot, sizeof(u64) * (size_t)K, cudaMemcpyDeviceToHost, st));
        RSC_CUDA_TRY(cudaMemcpyAsync(tot_c.data(), L.tot, sizeof(u64) * (size_t)K, cudaMemcpyDeviceToHost, st));
        RSC_CUDA_TRY(cudaStreamSynchronize(st));
        u64 M = 0;
        for (int64_t c = 0; c < K; ++c) M += tot_c[(size_t)c];
        const double gamma = p.gamma;
        double q = 0.0;
        for (int64_t c = 0; c < K && M > 0; ++c) {
            const double f = (double)tot_c[(size_t)c] / (double)M;
            q += (double)in_c[(size_t)c] / (double)M - gamma * f * f;
        }
        *modularity = q;
    }
    return RSC_OK;
}

}  // extern "C"
