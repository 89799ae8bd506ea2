// Large-basket tensor-core kernels, bf16 operands.
#include "k_basket_big.cuh"

namespace gbmc {
GBMC_INSTANTIATE_BIG(MC_BF16)
}  // namespace gbmc
