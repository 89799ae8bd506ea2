// Large-basket tensor-core kernels, fp8 operands.
#include "k_basket_big.cuh"

namespace gbmc {
GBMC_INSTANTIATE_BIG(MC_FP8E4M3)
}  // namespace gbmc
