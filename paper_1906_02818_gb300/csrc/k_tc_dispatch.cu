// Dispatch of the tensor-core basket kernels (instantiated per operand type
// in k_basket_tc_{bf16,fp16,fp8}.cu).
#include <cstdio>
#include <cstdlib>

#include "mc_kernels.cuh"

namespace gbmc {

template <int PREC, int SCHEME>
const void *basket_tc_select(const TcArgs &a, int *smem);
template <int PREC>
cudaError_t tc_prep(int d, const double *L, const double *sigma, double cfac, double sdt, double r, double dt,
                    int scheme, uint8_t *bimg, float *cs, float *drift, cudaStream_t s);

namespace {

constexpr int kTcThreads = 128;

template <int PREC>
const void *select_prec(const TcArgs &a, int *smem)
{
    return a.scheme == MC_LOG_EULER ? basket_tc_select<PREC, MC_LOG_EULER>(a, smem)
                                    : basket_tc_select<PREC, MC_EULER>(a, smem);
}

const void *select(int prec, const TcArgs &a, int *smem)
{
    switch (prec) {
    case MC_BF16: return select_prec<MC_BF16>(a, smem);
    case MC_FP16: return select_prec<MC_FP16>(a, smem);
    case MC_FP8E4M3: return select_prec<MC_FP8E4M3>(a, smem);
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
    // The same bound computed from the kernel's resources: registers (per-warp
    // allocation in units of 256), shared memory (static + dynamic + the
    // per-block reservation), threads, and TMEM (64 of 512 columns per CTA).
    cudaFuncAttributes fa;
    int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return nb > 8 ? 8 : nb;
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    int m = regs_sm / (warp_regs * (kTcThreads / 32));
    const int per_block_smem = static_cast<int>(fa.sharedSizeBytes) + smem + smem_res;
    m = per_block_smem > 0 && smem_sm / per_block_smem < m ? smem_sm / per_block_smem : m;
    m = thr_sm / kTcThreads < m ? thr_sm / kTcThreads : m;
    m = m > 8 ? 8 : m;
    if (std::getenv("GBMC_DEBUG"))
        std::fprintf(stderr, "[gbmc] tc occupancy: runtime %d, resources %d (regs %d, smem %d)\n", nb, m,
                     fa.numRegs, per_block_smem);
    // The runtime's answer can be lower than the resource bound for kernels
    // that use tensor memory; more CTAs than fit simply wait for a slot.
    return nb > m ? nb : m;
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
