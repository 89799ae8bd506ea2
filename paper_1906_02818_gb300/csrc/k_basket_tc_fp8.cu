// Tensor-core basket kernels, fp8 operands.
#include "k_basket_tc.cuh"

namespace gbmc {
GBMC_INSTANTIATE_TC(MC_FP8E4M3)
}  // namespace gbmc
