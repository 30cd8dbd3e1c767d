// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "rsc.h"

namespace rsc {

// Names an entry point's span in profiler timelines (an NVTX range, pushed on
// entry and popped on every return; nothing is recorded unless a profiler is
// attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define RSC_TRACE(name) ::rsc::TraceRange rsc_trace_range_(name)

// ---------------------------------------------------------------- host side

// Thread-local error message, returned by rsc_last_error().
void set_error(const char *fmt, ...);
rsc_status fail(rsc_status st, const char *fmt, ...);

#define RSC_CUDA_TRY(expr)                                                             \
    do {                                                                               \
        cudaError_t rsc_e_ = (expr);                                                   \
        if (rsc_e_ != cudaSuccess)                                                     \
            return ::rsc::fail(RSC_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,           \
                               cudaGetErrorString(rsc_e_), __FILE__, __LINE__);        \
    } while (0)

// Bump allocator over a caller-provided workspace.  With base == nullptr it
// only measures, so the same code computes the size and the layout.
struct Carve {
    char *base;
    size_t used = 0;
    explicit Carve(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

// The first 256 bytes of every workspace hold the status word kernels write.
constexpr size_t kStatusBytes = 256;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int sm_count();   // multiprocessors of the current device (cached per device)

// ------------------------------------------------------------- device side

// Records the first failure in the workspace status word.
__device__ __forceinline__ void record_status(unsigned int *status, unsigned int code) {
    if (status) atomicCAS(status, 0u, code);
}

// Three-input minimum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Minimum of v[0 .. 8).
__device__ __forceinline__ float min8(const float *v) {
    return fmin3(fmin3(v[0], v[1], v[2]), fmin3(v[3], v[4], v[5]), fminf(v[6], v[7]));
}

template <int N>
__device__ __forceinline__ float min_of(const float (&v)[N]) {
    static_assert(N == 16 || N == 32, "chunk of 16 or 32");
    float m[6];
    m[0] = fmin3(v[0], v[1], v[2]);
    m[1] = fmin3(v[3], v[4], v[5]);
    m[2] = fmin3(v[6], v[7], v[8]);
    m[3] = fmin3(v[9], v[10], v[11]);
    m[4] = fmin3(v[12], v[13], v[14]);
    float r = fmin3(m[0], m[1], m[2]);
    r = fmin3(r, m[3], m[4]);
    r = fminf(r, v[15]);
    if constexpr (N == 32) {
        m[0] = fmin3(v[16], v[17], v[18]);
        m[1] = fmin3(v[19], v[20], v[21]);
        m[2] = fmin3(v[22], v[23], v[24]);
        m[3] = fmin3(v[25], v[26], v[27]);
        m[4] = fmin3(v[28], v[29], v[30]);
        float s = fmin3(m[0], m[1], m[2]);
        s = fmin3(s, m[3], m[4]);
        r = fmin3(r, s, v[31]);
    }
    return r;
}

}  // namespace rsc
