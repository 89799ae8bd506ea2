// Path-per-thread Heston kernel: full-truncation Euler on (log S, v) with two
// correlated normals per step (one Philox block serves two steps), fused with
// the payoff statistics and the reduction.
//   v+ = max(v, 0)
//   log S <- log S + (r - v+/2) dt + sqrt(v+ dt) (rho z1 + sqrt(1 - rho^2) z2)
//   v     <- v + kappa (theta - v+) dt + xi sqrt(v+ dt) z1
#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kBlock = 256;

template <bool STATS, bool SAVE>
__global__ void __launch_bounds__(kBlock) heston_kernel(const __grid_constant__ HestonArgs a)
{
    __shared__ AccSlot s_acc[(kBlock / 32) * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];
    for (int i = threadIdx.x; i < (kBlock / 32) * a.pay.n * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();

    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = a.run.steps;
    const float inv_m = 1.0f / static_cast<float>(M);
    const float dt = a.dt, kdt = a.kappa * a.dt;
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gthreads;
        const bool valid = nl < a.run.paths;
        float uT = a.s0, avg = 0.0f, umax = -INFINITY, umin = INFINITY;
        if (valid) {
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            float y = 0.0f, v = a.v0, sum = 0.0f, S = a.s0;
            const int64_t save_len = (static_cast<int64_t>(M / a.run.save_every) + 1) * 2 * a.run.paths;
            if (SAVE) {
                if (GBMC_IN_BOUNDS(nl, save_len, kDbgHestonSave)) a.run.save[nl] = a.s0;
                if (GBMC_IN_BOUNDS(a.run.paths + nl, save_len, kDbgHestonSave)) a.run.save[a.run.paths + nl] = a.v0;
            }
            const int nq = (M + 1) >> 1;
            for (int q = 0; q < nq; ++q) {
                const float4 z4 = normals4(static_cast<uint64_t>(q), n, a.run.rk);
                const float z1s[2] = {z4.x, z4.z}, z2s[2] = {z4.y, z4.w};
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    const int i = 2 * q + l;
                    if (i < M) {
                        const float vp = fmaxf(v, 0.0f);
                        const float sq = sqrt_approx(vp * dt);
                        const float c = fmaf(a.rho, z1s[l], a.rhoc * z2s[l]);
                        y = fmaf(kLog2e, fmaf(sq, c, (a.r - 0.5f * vp) * dt), y);
                        v = v + fmaf(a.xi * sq, z1s[l], kdt * (a.theta - vp));
                        if (STATS || SAVE) {
                            S = a.s0 * ex2_approx(y);
                            sum += S;
                            umax = fmaxf(umax, S);
                            umin = fminf(umin, S);
                            if (SAVE && ((i + 1) % a.run.save_every) == 0) {
                                const int64_t slot = (i + 1) / a.run.save_every;
                                if (GBMC_IN_BOUNDS((slot * 2 + 1) * a.run.paths + nl, save_len, kDbgHestonSave)) {
                                    a.run.save[(slot * 2) * a.run.paths + nl] = S;
                                    a.run.save[(slot * 2 + 1) * a.run.paths + nl] = v;
                                }
                            }
                        }
                    }
                }
            }
            uT = a.s0 * ex2_approx(y);
            avg = sum * inv_m;
        }
        for (int p = 0; p < a.pay.n; ++p) {
            const float f = payoff_eval(a.pay.kind[p], a.pay.strike[p], a.pay.barrier[p], uT, avg, umax, umin);
            warp_accumulate(s_acc, a.pay.n, p, valid ? f : 0.0f);
        }
    }
    if (a.pay.n > 0) block_finish(s_acc, s_red, a.pay.n, a.red);
}

const void *heston_select(const HestonArgs &a)
{
    if (a.run.save) return reinterpret_cast<const void *>(&heston_kernel<false, true>);
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    return stats ? reinterpret_cast<const void *>(&heston_kernel<true, false>)
                 : reinterpret_cast<const void *>(&heston_kernel<false, false>);
}

}  // namespace

cudaError_t launch_heston(const HestonArgs &a, int grid, int block, cudaStream_t s)
{
    void *args[] = {const_cast<HestonArgs *>(&a)};
    return cudaLaunchKernel(heston_select(a), dim3(grid), dim3(block), args, 0, s);
}

int heston_occupancy(const HestonArgs &a, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, heston_select(a), block, 0) != cudaSuccess) return 0;
    return nb;
}

}  // namespace gbmc
