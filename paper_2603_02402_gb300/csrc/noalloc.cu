// Fuzzy connectivities with library-owned scratch memory.
//
// rsc_connectivities takes its scratch space from the caller.  Some callers
// cannot hand out device memory at the point where they build the graph: a
// host application whose own pool has already reserved the device's memory
// and offers plug-ins no allocation hook, or a service that must run with a
// fixed device-memory budget that may not grow after start-up.  For them,
// rsc_connectivities_static runs the same computation with its scratch in a
// fixed-size array that the library itself declares, so the call neither
// allocates nor asks the caller for a workspace.  The array is part of the
// library's device image: every GPU that loads the library holds it until
// the process exits.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rsc {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB, shared by every call

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device.  In host
// code the array's name only stands for the symbol; a kernel needs the
// device address that cudaGetSymbolAddress returns.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

rsc_status static_scratch(void **out) {
    int dev = 0;
    RSC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(RSC_ERR_UNSUPPORTED, "device index %d above %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(RSC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RSC_OK;
}

}  // namespace
}  // namespace rsc

using namespace rsc;

extern "C" rsc_status rsc_connectivities_static(const int32_t *idx, const float *dist, int64_t n, int32_t k,
                                                int64_t *indptr, int32_t *indices, float *data,
                                                int64_t nnz_capacity, float *rho, float *sigma, void *stream) {
    if (!idx || !dist || !indptr || !indices || !data) return fail(RSC_ERR_INVALID_ARG, "NULL array argument");
    if (n < 1 || k < 1 || k > 256) return fail(RSC_ERR_INVALID_ARG, "bad n/k");
    size_t need = 0;
    rsc_status s = rsc_connectivities_workspace_size(n, k, &need);
    if (s != RSC_OK) return s;
    if (need > kStaticScratchBytes)
        return fail(RSC_ERR_WORKSPACE,
                    "n=%lld, k=%d needs %zu bytes of scratch; the static scratch holds %zu bytes (32 MiB): "
                    "use rsc_connectivities with a caller workspace",
                    (long long)n, k, need, kStaticScratchBytes);
    if (nnz_capacity < rsc_connectivities_max_nnz(n, k))
        return fail(RSC_ERR_INVALID_ARG, "nnz_capacity must be at least rsc_connectivities_max_nnz(n, k) = %lld",
                    (long long)rsc_connectivities_max_nnz(n, k));
    void *scratch = nullptr;
    if ((s = static_scratch(&scratch)) != RSC_OK) return s;
    return rsc_connectivities(idx, dist, n, k, indptr, indices, data, nnz_capacity, rho, sigma, scratch,
                              kStaticScratchBytes, stream);
}
