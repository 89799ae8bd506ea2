// Dispatch, factor preparation and launchers of the two-level estimator's
// correction kernel (k_mlmc.cuh; instantiated per operand type in
// k_mlmc_{bf16,fp16,fp8}.cu).
#include "k_mlmc.cuh"

namespace gbmc {

extern template const void *mlmc_select_prec<MC_BF16>(const MlmcArgs &a);
extern template const void *mlmc_select_prec<MC_FP16>(const MlmcArgs &a);
extern template const void *mlmc_select_prec<MC_FP8E4M3>(const MlmcArgs &a);

namespace {

const void *select(int prec, const MlmcArgs &a)
{
    switch (prec) {
    case MC_BF16: return mlmc_select_prec<MC_BF16>(a);
    case MC_FP16: return mlmc_select_prec<MC_FP16>(a);
    case MC_FP8E4M3: return mlmc_select_prec<MC_FP8E4M3>(a);
    default: return nullptr;
    }
}

// Dequantised factor entries as the tensor-core factor tile holds them, in
// units of the scaled row (Lq[n][k] = round(L[n][k] s_n)), and the column
// scales cs_n = c sqrt(dt) sigma_n / s_n; s_n = 448 / max_k |L[n][k]| for
// E4M3, c sqrt(dt) sigma_n for BF16 (so cs_n = 1), 1 for FP16.  Packed lower
// triangle, rows of width 64.
template <int PREC>
__global__ void mlmc_prep_kernel(int d, const double *L, const double *sigma, double cfac, double sdt, float *Lq,
                                 float *csq)
{
    const int nrow = threadIdx.x;
    if (nrow >= kD) return;
    double amax = 0.0;
    for (int k = 0; k <= nrow && k < d; ++k) amax = fmax(amax, fabs(nrow < d ? L[static_cast<int64_t>(nrow) * d + k] : 0.0));
    const double colscale = nrow < d ? cfac * sdt * sigma[nrow] : 0.0;  // sigma_n = 0: a zero row
    const double s = (PREC == MC_FP8E4M3 && amax > 0.0) ? 448.0 / amax : (PREC == MC_BF16 ? colscale : 1.0);
    for (int k = 0; k <= nrow; ++k) {
        const double v = (nrow < d && k < d) ? L[static_cast<int64_t>(nrow) * d + k] * s : 0.0;
        Lq[nrow * (nrow + 1) / 2 + k] = round_operand<PREC>(static_cast<float>(v));
    }
    csq[nrow] = nrow < d ? (PREC == MC_BF16 ? 1.0f : static_cast<float>(cfac * sdt * sigma[nrow] / s)) : 0.0f;
}

}  // namespace

cudaError_t launch_mlmc_prep(int prec, int d, const double *L, const double *sigma, double cfac, double sdt,
                             float *Lq, float *csq, cudaStream_t s)
{
    switch (prec) {
    case MC_BF16: mlmc_prep_kernel<MC_BF16><<<1, kD, 0, s>>>(d, L, sigma, cfac, sdt, Lq, csq); break;
    case MC_FP16: mlmc_prep_kernel<MC_FP16><<<1, kD, 0, s>>>(d, L, sigma, cfac, sdt, Lq, csq); break;
    case MC_FP8E4M3: mlmc_prep_kernel<MC_FP8E4M3><<<1, kD, 0, s>>>(d, L, sigma, cfac, sdt, Lq, csq); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mlmc_coupled(int prec, const MlmcArgs &a, const MlmcConst &c, int grid, cudaStream_t s)
{
    const void *f = select(prec, a);
    if (!f) return cudaErrorInvalidValue;
    void *args[] = {const_cast<MlmcArgs *>(&a), const_cast<MlmcConst *>(&c)};
    return cudaLaunchKernel(f, dim3(grid), dim3(kBlock), args, 0, s);
}

int mlmc_occupancy(int prec, const MlmcArgs &a)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select(prec, a), kBlock, 0) != cudaSuccess) return 0;
    return nb;
}

int mlmc_block() { return kBlock; }
int mlmc_paths_per_block() { return kHalf; }

}  // namespace gbmc
