// Dispatch of the large-basket kernels: tensor-core variants (per operand
// type, k_basket_big_*.cu) and the FP32 variant (k_basket_wide.cu).
#include "mc_kernels.cuh"

namespace gbmc {

template <int PREC>
const void *basket_big_fn();
template <int PREC>
int basket_big_smem();
template <int PREC>
cudaError_t big_prep(int d, const double *L, const double *sigma, double cfac, double sdt, double r, double dt, int M,
                     uint8_t *bimg, float *cs, float *mdrift, float *vscale, cudaStream_t s);
const void *basket_wide_fn(int D);
int basket_wide_block();
int wide_width(int d);
size_t wide_smem(int D);

namespace {

constexpr int kBigThreads = 576;

const void *select(int prec, int d, int *smem, int *threads)
{
    *threads = kBigThreads;
    switch (prec) {
    case MC_BF16: *smem = basket_big_smem<MC_BF16>(); return basket_big_fn<MC_BF16>();
    case MC_FP16: *smem = basket_big_smem<MC_FP16>(); return basket_big_fn<MC_FP16>();
    case MC_FP8E4M3: *smem = basket_big_smem<MC_FP8E4M3>(); return basket_big_fn<MC_FP8E4M3>();
    default: {
        const int D = wide_width(d);
        *smem = static_cast<int>(wide_smem(D));
        *threads = basket_wide_block();
        return basket_wide_fn(D);
    }
    }
}

}  // namespace

// 4 row blocks x 8 panels of 128 x 64 operand chunks
size_t big_bimg_bytes(int prec) { return static_cast<size_t>(32) * (prec == MC_FP8E4M3 ? 8192 : 16384); }

cudaError_t launch_basket_big(int prec, const BigArgs &a, int grid, cudaStream_t s)
{
    int smem = 0, threads = 0;
    const void *fn = select(prec, a.d, &smem, &threads);
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {const_cast<BigArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, static_cast<size_t>(smem), s);
}

// One CTA per SM for both variants (tensor cores: the accumulator takes all
// of TMEM; FP32: the normals and factor chunks take most of shared memory),
// at most one per tile (128 paths, resp. 64 paths).
int basket_big_grid(int prec, int64_t paths)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const int rows = prec != MC_FP32 ? 128 : 64;
    const int64_t tiles = (paths + rows - 1) / rows;
    return static_cast<int>(tiles < sms ? tiles : sms);
}

cudaError_t launch_big_prep(int prec, int d, const double *L, const double *sigma, double cfac, double sdt, double r,
                            double dt, int M, uint8_t *bimg, float *cs, float *mdrift, float *vscale, cudaStream_t s)
{
    switch (prec) {
    case MC_BF16: return big_prep<MC_BF16>(d, L, sigma, cfac, sdt, r, dt, M, bimg, cs, mdrift, vscale, s);
    case MC_FP16: return big_prep<MC_FP16>(d, L, sigma, cfac, sdt, r, dt, M, bimg, cs, mdrift, vscale, s);
    case MC_FP8E4M3: return big_prep<MC_FP8E4M3>(d, L, sigma, cfac, sdt, r, dt, M, bimg, cs, mdrift, vscale, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbmc
