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
#include "common.cuh"
#include "kernels.h"

namespace rsc {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB, shared by every call

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current context.  In host code
// the array's name only stands for the symbol; a kernel needs the device
// address that cudaGetSymbolAddress returns.  The address belongs to the
// context that loaded the module, so it is looked up on every call (a host
// query, no GPU work): a cached value would go stale after cudaDeviceReset
// or when the caller makes another context current on the same device.
rsc_status static_scratch(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail(RSC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    *out = p;
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
