// Tensor-core basket kernels, fp16 operands.
#include "k_basket_tc.cuh"

namespace gbmc {
GBMC_INSTANTIATE_TC(MC_FP16)
}  // namespace gbmc
