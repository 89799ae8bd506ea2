// Correction-level kernels of the two-level estimator, bf16 operand arithmetic.
#include "k_mlmc.cuh"

namespace gbmc {
template const void *mlmc_select_prec<MC_BF16>(const MlmcArgs &a);
}  // namespace gbmc
