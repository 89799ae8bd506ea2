// Correction level of the two-level precision estimator (Sec. V: a
// low-precision simulation as a companion estimator whose bias is identified
// with few samples and corrected, after Giles' multilevel Monte Carlo):
//   E[P_fp32] = E[P_q] + E[P_fp32 - P_q],
// the first term from many tensor-core paths (mc_plan_execute with BF16 /
// FP16 / E4M3 operands), the second from fewer paths simulated twice on the
// same normals by this kernel:
//   pass 1: the FP32 contraction (dW = Lhat z, the FP32 basket kernel's step,
//           in the same packed FP32x2 FMAs);
//   pass 2: the tensor-core arithmetic with FP32 accumulation: normals rounded
//           to the operand type (E4M3 scaled per step by 448 / max|z| of the
//           path's row and dequantised by max|z| / 448), the factor rounded as
//           the tensor-core factor tile (rows scaled by s_n, column scale
//           cs_n = c sqrt(dt) sigma_n / s_n folded after the sum).
// Per path and payoff it accumulates f_fp32 - f_q, f_fp32 and f_q.  A block
// carries 64 paths at a time: its first two warps run them in FP32, the other
// two in the rounded arithmetic (twice the warps for the few paths this
// level takes), and the rounded payoffs pass through shared memory; d <= 64
// padded to 64.  The kernels are instantiated per
// operand type in k_mlmc_{bf16,fp16,fp8}.cu; k_mlmc.cu holds the dispatch,
// the factor preparation and the launchers.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kD = 64;
constexpr int kBlock = 128;
constexpr int kHalf = kBlock / 2;  // paths a block carries at a time

template <int PREC>
__device__ __forceinline__ float round_operand(float v)
{
    if (PREC == MC_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    if (PREC == MC_FP16) return __half2float(__float2half_rn(v));
    uint16_t pr;  // E4M3 (saturating) in the low byte, then back through f16x2 (exact)
    uint32_t h2;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(pr) : "f"(0.0f), "f"(v));
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(pr));
    return __half2float(__ushort_as_half(static_cast<unsigned short>(h2 & 0xFFFFu)));
}

struct PathOut {
    float uT, avg, umax, umin;
};

// One path of the correlated GBM basket; quant selects the tensor-core
// operand arithmetic (pass 2) instead of the FP32 contraction (pass 1).  One
// out-of-line copy serves both passes: the two fully unrolled copies did not
// fit the instruction cache together (no_instruction stalls).
template <int PREC, int SCHEME, bool STATS>
__device__ __noinline__ PathOut simulate(const MlmcArgs &a, const MlmcConst &c, uint64_t n, bool quant)
{
    const int M = a.run.steps, d = a.d;
    NormalReader rd;
    rd.init(n, a.run.rk);
    float x[kD];
#pragma unroll
    for (int j = 0; j < kD; ++j) x[j] = (SCHEME == MC_LOG_EULER) ? 0.0f : c.s0[j];
    float sum = 0.0f, umax = -INFINITY, umin = INFINITY;
    for (int i = 0; i < M; ++i) {
        // E4M3: the row scale needs the step's largest |z| first
        float sz = 1.0f, deq = 1.0f;
        if (quant && PREC == MC_FP8E4M3) {
            float amax = 0.0f;
            for (int k = 0; k < d; ++k) amax = fmaxf(amax, fabsf(rd.get(static_cast<uint64_t>(i) * d + k)));
            if (amax > 0.0f) {
                sz = 448.0f / amax;
                deq = amax / 448.0f;
            }
        }
        // dW = Lhat z column by column in packed FP32x2 FMAs over row pairs
        // (each lane an ordinary fma, the columns in order per element)
        f32x2 acc2[kD / 2];
#pragma unroll
        for (int q = 0; q < kD / 2; ++q) acc2[q] = pack2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            float z = k < d ? rd.get(static_cast<uint64_t>(i) * d + k) : 0.0f;
            if (quant) z = round_operand<PREC>(PREC == MC_FP8E4M3 ? z * sz : z);
            const f32x2 z2 = pack2(z, z);
#pragma unroll
            for (int q = k / 2; q < kD / 2; ++q)
                acc2[q] = ffma2(quant ? c.Lqp[basket_pair_base(kD, k) + q - k / 2] : c.Lp[basket_pair_base(kD, k) + q - k / 2],
                                z2, acc2[q]);
        }
        float u = 0.0f;
#pragma unroll
        for (int j = 0; j < kD; ++j) {
            const float aj = (j & 1) ? hi_of(acc2[j >> 1]) : lo_of(acc2[j >> 1]);
            const float dw = quant ? c.csq[j] * (aj * deq) : aj;
            if (SCHEME == MC_LOG_EULER) {
                x[j] += c.drift[j] + dw;
                if (STATS) u = fmaf(c.ws0[j], ex2_approx(x[j]), u);
            } else {
                x[j] = fmaf(x[j], c.drift[j] + dw, x[j]);
                if (STATS) u = fmaf(c.w[j], x[j], u);
            }
        }
        if (STATS) {
            sum += u;
            umax = fmaxf(umax, u);
            umin = fminf(umin, u);
        }
    }
    float uT = 0.0f;
#pragma unroll
    for (int j = 0; j < kD; ++j) uT = (SCHEME == MC_LOG_EULER) ? fmaf(c.ws0[j], ex2_approx(x[j]), uT) : fmaf(c.w[j], x[j], uT);
    return PathOut{uT, sum / static_cast<float>(M), umax, umin};
}

template <int PREC, int SCHEME, bool STATS>
__global__ void __launch_bounds__(kBlock) mlmc_coupled_kernel(const __grid_constant__ MlmcArgs a, const MlmcConst c)
{
    __shared__ AccSlot s_acc[(kBlock / 32) * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];
    __shared__ float s_fq[kMlmcMaxPayoffs][kHalf];
    const int np = a.pay.n, nv = 3 * np;
    for (int i = threadIdx.x; i < (kBlock / 32) * nv * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();
    const int half = threadIdx.x / kHalf, lt = threadIdx.x % kHalf;  // half: warp-uniform
    const int64_t gpaths = static_cast<int64_t>(gridDim.x) * kHalf;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * kHalf + lt;
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gpaths;
        const bool valid = nl < a.run.paths;
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + (valid ? nl : 0));
        const PathOut o = simulate<PREC, SCHEME, STATS>(a, c, n, half != 0);
        float f[kMlmcMaxPayoffs];
#pragma unroll
        for (int p = 0; p < kMlmcMaxPayoffs; ++p)
            f[p] = p < np ? payoff_eval(a.pay.kind[p], a.pay.strike[p], a.pay.barrier[p], o.uT, o.avg, o.umax, o.umin)
                          : 0.0f;
        if (half) {
#pragma unroll
            for (int p = 0; p < kMlmcMaxPayoffs; ++p)
                if (p < np) s_fq[p][lt] = f[p];
        }
        __syncthreads();
        if (!half) {
#pragma unroll
            for (int p = 0; p < kMlmcMaxPayoffs; ++p) {
                if (p < np) {
                    const float fe = f[p], fq = s_fq[p][lt];
                    warp_accumulate(s_acc, nv, p, valid ? fe - fq : 0.0f);
                    warp_accumulate(s_acc, nv, np + p, valid ? fe : 0.0f);
                    warp_accumulate(s_acc, nv, 2 * np + p, valid ? fq : 0.0f);
                }
            }
        }
        __syncthreads();  // the rounded payoffs are read before the next paths write theirs
    }
    block_finish(s_acc, s_red, nv, a.red);
}

template <int PREC, int SCHEME, bool STATS>
const void *fn() { return reinterpret_cast<const void *>(&mlmc_coupled_kernel<PREC, SCHEME, STATS>); }

}  // namespace

template <int PREC>
const void *mlmc_select_prec(const MlmcArgs &a)
{
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    if (a.scheme == MC_LOG_EULER) return stats ? fn<PREC, MC_LOG_EULER, true>() : fn<PREC, MC_LOG_EULER, false>();
    return stats ? fn<PREC, MC_EULER, true>() : fn<PREC, MC_EULER, false>();
}

}  // namespace gbmc
