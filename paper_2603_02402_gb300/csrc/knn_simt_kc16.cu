// FP32 SIMT candidate search, KC = 16 (all DP variants).
#include "knn_simt.cuh"

namespace rsc {
RSC_DEFINE_SIMT_KC(16)
}  // namespace rsc
