// FP32 basket kernels, width 64, log-Euler scheme.
#define GBMC_BASKET_IMPL
#include "k_basket.cuh"

namespace gbmc {
GBMC_INSTANTIATE_BASKET(64, MC_LOG_EULER)
}  // namespace gbmc
