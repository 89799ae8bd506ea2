// Large-basket tensor-core kernels, fp16 operands.
#include "k_basket_big.cuh"

namespace gbmc {
GBMC_INSTANTIATE_BIG(MC_FP16)
}  // namespace gbmc
