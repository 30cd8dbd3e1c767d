// Dispatch of the FP32 SIMT candidate search (kernel in knn_simt.cuh).
#include "knn_simt.cuh"

namespace rsc {

bool knn_simt_supported(int DP, int KC) {
    const bool dp_ok = DP >= 8 && DP <= 64 && DP % 8 == 0;
    const bool kc_ok = KC == 16 || KC == 32 || KC == 64;
    return dp_ok && kc_ok;
}

cudaError_t launch_knn_simt(const float *Y, const float *ny, int64_t n, int DP, int width, int KC,
                            int splits, int64_t split_len, int32_t *cand, cudaStream_t st) {
    if (width < DP - 7 || width > DP) return cudaErrorInvalidValue;
    switch (KC) {
        case 16: return launch_knn_simt_kc<16>(DP, Y, ny, n, width, splits, split_len, cand, st);
        case 32: return launch_knn_simt_kc<32>(DP, Y, ny, n, width, splits, split_len, cand, st);
        case 64: return launch_knn_simt_kc<64>(DP, Y, ny, n, width, splits, split_len, cand, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rsc
