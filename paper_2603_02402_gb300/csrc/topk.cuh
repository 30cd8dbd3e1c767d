// Per-thread bounded top-k for distance rows that one thread owns.
//
// Each thread keeps the KC smallest (key, column) pairs of its query row in
// registers, sorted ascending; the threshold is the KC-th key.  Values arrive
// in chunks of CH.  A chunk whose minimum is not below the threshold (the
// common case once the list has filled) costs one min tree and one compare.
// Otherwise the chunk's qualifying values are appended to a per-thread
// shared-memory buffer; the buffer is merged into the register list when it
// could overflow and at tile boundaries, so the costly sorted insertions of a
// warp's lanes run side by side rather than one lane at a time.
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
    __device__ __forceinline__ void insert(float v, int j) {
#pragma unroll
        for (int c = KC - 1; c > 0; --c) {
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

// Shared-memory candidate buffer of one thread: entry e lives at
// base[e * stride]; with stride = threads per block, lanes of a warp always
// hit distinct banks whatever their fill levels.
template <int KC, int CAP>
struct BufferedTopK {
    RowTopK<KC> list;
    float *bkey;
    int *bid;
    int stride;
    int cnt;

    __device__ __forceinline__ void init(float *keys, int *ids, int thread, int nthreads) {
        list.init();
        bkey = keys + thread;
        bid = ids + thread;
        stride = nthreads;
        cnt = 0;
    }

    __device__ __forceinline__ void flush() {
        for (int e = 0; e < cnt; ++e) {
            const float v = bkey[e * stride];
            if (v < list.thr()) list.insert(v, bid[e * stride]);
        }
        cnt = 0;
    }

    // Offer CH values of columns j0 .. j0 + CH - 1.
    template <int CH>
    __device__ __forceinline__ void offer(const float (&v)[CH], int j0) {
        static_assert(CH <= CAP, "buffer smaller than a chunk");
        const float m = min_of<CH>(v);
        if (m < list.thr()) {
            if (cnt > CAP - CH) flush();
            const float t = list.thr();
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                if (v[i] < t) {
                    bkey[cnt * stride] = v[i];
                    bid[cnt * stride] = j0 + i;
                    ++cnt;
                }
            }
        }
    }
};

}  // namespace rsc
