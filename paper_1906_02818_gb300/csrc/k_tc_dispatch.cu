// Dispatch of the tensor-core basket kernels (instantiated per operand type
// in k_basket_tc_{bf16,fp16,fp8}.cu).
#include "mc_kernels.cuh"

namespace gbmc {

template <int PREC, int SCHEME>
const void *basket_tc_select(const TcArgs &a);
template <int PREC>
int basket_tc_smem();
template <int PREC>
cudaError_t tc_prep(int d, const double *L, const double *sigma, double cfac, double sdt, double r, double dt,
                    int scheme, uint8_t *bimg, float *cs, float *drift, cudaStream_t s);

namespace {

constexpr int kTcThreads = 128;

template <int PREC>
const void *select_prec(const TcArgs &a)
{
    return a.scheme == MC_LOG_EULER ? basket_tc_select<PREC, MC_LOG_EULER>(a) : basket_tc_select<PREC, MC_EULER>(a);
}

const void *select(int prec, const TcArgs &a, int *smem)
{
    switch (prec) {
    case MC_BF16: *smem = basket_tc_smem<MC_BF16>(); return select_prec<MC_BF16>(a);
    case MC_FP16: *smem = basket_tc_smem<MC_FP16>(); return select_prec<MC_FP16>(a);
    case MC_FP8E4M3: *smem = basket_tc_smem<MC_FP8E4M3>(); return select_prec<MC_FP8E4M3>(a);
    default: *smem = 0; return nullptr;
    }
}

}  // namespace

int tc_bimg_bytes(int prec) { return prec == MC_FP8E4M3 ? 64 * 64 : 64 * 64 * 2; }

cudaError_t launch_basket_tc(int prec, const TcArgs &a, const TcConst &c, int grid, cudaStream_t s)
{
    int smem = 0;
    const void *fn = select(prec, a, &smem);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<TcArgs *>(&a), const_cast<TcConst *>(&c)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), args, static_cast<size_t>(smem), s);
}

int basket_tc_occupancy(int prec, const TcArgs &a)
{
    int smem = 0;
    const void *fn = select(prec, a, &smem);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTcThreads, smem) != cudaSuccess) return 0;
    // every resident CTA holds 64 TMEM columns of the SM's 512
    return nb > 8 ? 8 : nb;
}

cudaError_t launch_tc_prep(int prec, int d, const double *L, const double *sigma, double c, double sdt,
                           double r, double dt, int scheme, uint8_t *bimg, float *cs, float *drift,
                           cudaStream_t s)
{
    switch (prec) {
    case MC_BF16: return tc_prep<MC_BF16>(d, L, sigma, c, sdt, r, dt, scheme, bimg, cs, drift, s);
    case MC_FP16: return tc_prep<MC_FP16>(d, L, sigma, c, sdt, r, dt, scheme, bimg, cs, drift, s);
    case MC_FP8E4M3: return tc_prep<MC_FP8E4M3>(d, L, sigma, c, sdt, r, dt, scheme, bimg, cs, drift, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbmc
