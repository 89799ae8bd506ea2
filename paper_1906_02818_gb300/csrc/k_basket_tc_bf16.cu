// Tensor-core basket kernels, bf16 operands.
#include "k_basket_tc.cuh"

namespace gbmc {
GBMC_INSTANTIATE_TC(MC_BF16)
}  // namespace gbmc
