// Correction-level kernels of the two-level estimator, fp8 operand arithmetic.
#include "k_mlmc.cuh"

namespace gbmc {
template const void *mlmc_select_prec<MC_FP8E4M3>(const MlmcArgs &a);
}  // namespace gbmc
