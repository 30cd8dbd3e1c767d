// Per-thread bounded top-k for distance rows that one thread owns.
//
// Each thread keeps the KC smallest (key, column) pairs of its query row in
// registers, sorted ascending; the threshold is the KC-th key.  Values arrive
// in chunks of 16.  A chunk whose minimum is not below the threshold (the
// common case once the list has filled) costs a 3-input min tree and one
// compare.  Otherwise the chunk's qualifying values are appended to a
// per-thread shared-memory buffer, merged into the register list only when
// some lane's buffer could overflow (and at the end of a row's scan).
#pragma once

#include <math.h>

#include "common.cuh"

namespace rsc {

template <int KC>
struct RowTopK {
    float key[KC];
    int id[KC];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            key[c] = INFINITY;
            id[c] = -1;
        }
    }
    __device__ __forceinline__ float thr() const { return key[KC - 1]; }

    // Sorted insertion; strict '<' keeps the earlier of equal keys first.
    // Caller guarantees v < thr().
    __device__ __forceinline__ void insert(float v, int j) { insert_prefix<KC>(v, j); }

    // Sorted insertion into the first P entries only (the rest untouched):
    // for lists of which only the best P are wanted.  Caller guarantees
    // v < key[P - 1].
    template <int P>
    __device__ __forceinline__ void insert_prefix(float v, int j) {
#pragma unroll
        for (int c = P - 1; c > 0; --c) {
            const bool lt_prev = v < key[c - 1];
            const bool lt_cur = v < key[c];
            const float nk = lt_prev ? key[c - 1] : (lt_cur ? v : key[c]);
            const int ni = lt_prev ? id[c - 1] : (lt_cur ? j : id[c]);
            key[c] = nk;
            id[c] = ni;
        }
        if (v < key[0]) {
            key[0] = v;
            id[0] = j;
        }
    }
};

// Shared-memory candidate buffer of one thread: keys of entry e at
// keys[e * STRIDE], ids at keys[(CAP + e) * STRIDE] (the id block follows the
// key block); with STRIDE = threads per block, lanes of a warp always hit
// distinct banks whatever their fill levels.  The buffer is addressed by its
// 32-bit shared-window address, which keeps the register cost at one word.
//
// All calls are warp-synchronous (every lane of the warp calls them
// together): the decision to merge buffers into the register lists is taken
// for the whole warp, so the lanes' sorted insertions run side by side
// instead of one lane at a time.  A lane's threshold is only refreshed at
// merges; a stale (higher) threshold admits extra candidates but never drops
// one of the KC best, because thresholds only decrease.
//
// SHORT > 0: when `shortl` is set only the best SHORT entries are wanted, so
// the filtering threshold is the SHORT-th key and insertions shift only the
// first SHORT entries.
template <int KC, int CAP, int STRIDE, int SHORT = 0>
struct BufferedTopK {
    static constexpr uint32_t kEntry = 4u * STRIDE;          // bytes between entries
    static constexpr uint32_t kIds = 4u * STRIDE * CAP;      // bytes from keys to ids
    RowTopK<KC> list;
    uint32_t sbase;   // shared address of this thread's key 0
    int cnt;
    bool shortl;

    // `keys`: the block's buffer (2 * CAP * STRIDE words); thread < STRIDE.
    __device__ __forceinline__ void init(float *keys, int thread) {
        list.init();
        sbase = (uint32_t)__cvta_generic_to_shared(keys + thread);
        cnt = 0;
        shortl = false;
    }

    __device__ __forceinline__ void reset() {
        list.init();
        cnt = 0;
    }

    // Empty list that accepts only values <= m: every slot holds the next
    // float above m (id -1).  Correct when at least KC values <= m will be
    // offered before the list is read: they displace every such slot, and
    // larger values could never have been among the KC smallest.
    __device__ __forceinline__ void start_below(float m) {
        const float s = nextafterf(m, INFINITY);
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            list.key[c] = s;
            list.id[c] = -1;
        }
    }

    __device__ __forceinline__ float bound() const {
        if constexpr (SHORT > 0 && SHORT < KC) return shortl ? list.key[SHORT - 1] : list.key[KC - 1];
        else return list.thr();
    }

    __device__ __forceinline__ void put(int e, float v, int j) const {
        const uint32_t a = sbase + (uint32_t)e * kEntry;
        asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(a + kIds), "r"(j) : "memory");
    }
    __device__ __forceinline__ float key_at(int e) const {
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(sbase + (uint32_t)e * kEntry) : "memory");
        return v;
    }
    __device__ __forceinline__ int id_at(int e) const {
        int j;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(j) : "r"(sbase + (uint32_t)e * kEntry + kIds) : "memory");
        return j;
    }

    // Merge every lane's buffer into its list (warp-synchronous).
    __device__ __forceinline__ void flush() {
        const int rounds = __reduce_max_sync(0xffffffffu, cnt);
        for (int e = 0; e < rounds; ++e) {
            if (e < cnt) {
                const float v = key_at(e);
                if (v < bound()) {
                    if constexpr (SHORT > 0 && SHORT < KC) {
                        if (shortl) list.template insert_prefix<SHORT>(v, id_at(e));   // warp-uniform per item
                        else list.insert(v, id_at(e));
                    } else {
                        list.insert(v, id_at(e));
                    }
                }
            }
        }
        cnt = 0;
    }

    template <int G>
    __device__ __forceinline__ void append(const float *v, int j0, float t) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (v[i] < t) {
                put(cnt, v[i], j0 + i);
                ++cnt;
            }
        }
    }

    // Offer 16 values of columns j0 .. j0 + 15 whose two minima of 8 are
    // known (warp-synchronous).
    __device__ __forceinline__ void offer16m(const float *v, float m_lo, float m_hi, int j0) {
        static_assert(CAP >= 16, "buffer smaller than a chunk");
        const bool hit = fminf(m_lo, m_hi) < bound();
        if (__any_sync(0xffffffffu, hit)) {
            if (__any_sync(0xffffffffu, hit && cnt > CAP - 16)) flush();
            const float t = bound();
            if (m_lo < t) append<8>(v, j0, t);
            if (m_hi < t) append<8>(v + 8, j0 + 8, t);
        }
    }

    // Offer CH = 16 values of columns j0 .. j0 + 15 (warp-synchronous).
    __device__ __forceinline__ void offer16(const float (&v)[16], int j0) {
        static_assert(CAP >= 16, "buffer smaller than a chunk");
        const float m_lo = fmin3(fmin3(v[0], v[1], v[2]), fmin3(v[3], v[4], v[5]), fminf(v[6], v[7]));
        const float m_hi = fmin3(fmin3(v[8], v[9], v[10]), fmin3(v[11], v[12], v[13]), fminf(v[14], v[15]));
        const bool hit = fminf(m_lo, m_hi) < bound();
        if (__any_sync(0xffffffffu, hit)) {
            if (__any_sync(0xffffffffu, hit && cnt > CAP - 16)) flush();
            const float t = bound();
            if (m_lo < t) append<8>(v, j0, t);
            if (m_hi < t) append<8>(v + 8, j0 + 8, t);
        }
    }
};

}  // namespace rsc
