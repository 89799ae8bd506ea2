// FP32 correlated-basket path kernel (the multivariate Euler-Maruyama scheme
// of Sec. II.A.2), instantiated per basket width D in separate translation
// units so that they compile in parallel.  The contraction dW = Lhat z runs
// in packed FP32x2 FMAs (fma.rn.f32x2: two assets per instruction, each lane
// an ordinary FP32 fma) with the factor's column pairs in the
// launch-parameter block (constant bank) as 64-bit operands; the state is
// held as asset pairs.  A scalar FMA with a 32-bit constant-bank operand
// sustains a fraction of the FMA pipe's rate on this part; the 64-bit pair
// operand carries two factor entries per instruction.
//
// Large runs launch one block per SM, of up to 640 threads (trimmed to whole
// warps so that the rounds of paths fill every SM), whose warps meet at a
// block barrier after every four columns of a step, so that all warps of an
// SM read the same few hundred bytes of the factor at a time; small runs
// launch blocks of 128 (more SMs busy).  Either way every thread runs every
// step (threads past the last path compute a path whose results are
// dropped), which keeps the barriers uniform.  A factor staged in shared
// memory instead was slower: each 16-byte shared load costs four cycles of
// the shared-memory port, a quarter of the rate the packed FMAs need.
#pragma once

#include "mc_kernels.cuh"

namespace gbmc {

// Kernel entry for width D and the given scheme, chosen by the flags of `a`
// (explicitly instantiated in k_basket_*.cu).
template <int D, int SCHEME>
const void *basket_select_scheme(const BasketArgs &a);

#ifdef GBMC_BASKET_IMPL
namespace basket_detail {

constexpr int kBlock = 640;        // slots of the reduction (at most 20 warps)
constexpr int kLaunchBlock = 640;  // the largest launch block (mc_api: up to 640, or 128); 20 warps per SM

__device__ __forceinline__ float elem(const f32x2 *v, int j) { return (j & 1) ? hi_of(v[j >> 1]) : lo_of(v[j >> 1]); }

struct Stats {
    float sum, umax, umin;
    __device__ __forceinline__ void init() { sum = 0.0f; umax = -INFINITY; umin = INFINITY; }
    __device__ __forceinline__ void add(float u) { sum += u; umax = fmaxf(umax, u); umin = fminf(umin, u); }
};

__device__ __forceinline__ void accumulate_payoffs(AccSlot *s_acc, const PayoffSet &pay, bool valid,
                                                   float uT, float avg, const Stats &st)
{
    for (int p = 0; p < pay.n; ++p) {
        float f = payoff_eval(pay.kind[p], pay.strike[p], pay.barrier[p], uT, avg, st.umax, st.umin);
        warp_accumulate(s_acc, pay.n, p, valid ? f : 0.0f);
    }
}

// ------------------------------ FP32 basket -------------------------------
template <int D, int SCHEME, bool STATS, bool SAVE, bool EXACT>
__global__ void __launch_bounds__(kLaunchBlock, 1) basket_fp32_kernel(const __grid_constant__ BasketArgs a, const BasketConst<D> c)
{
    __shared__ AccSlot s_acc[(kBlock / 32) * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];
    for (int i = threadIdx.x; i < (kBlock / 32) * a.pay.n * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();

    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = a.run.steps, d = a.d;
    const float inv_m = 1.0f / static_cast<float>(M);
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gthreads;
        const bool valid = nl < a.run.paths;
        float uT = 0.0f, avg = 0.0f;
        Stats st;
        st.init();
        if (valid || !SAVE) {  // every thread steps (block barriers below) unless it writes paths
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            constexpr int H = D / 2;
            f32x2 x[H];  // asset pairs; log-Euler: log2(S_a / S0_a); Euler: S_a
#pragma unroll
            for (int q = 0; q < H; ++q)
                x[q] = (SCHEME == MC_LOG_EULER) ? pack2(0.0f, 0.0f) : pack2(c.s0[2 * q], c.s0[2 * q + 1]);
            const int64_t save_len = (static_cast<int64_t>(M / a.run.save_every) + 1) * d * a.run.paths;
            if (SAVE) {
                for (int j = 0; j < d; ++j)
                    if (GBMC_IN_BOUNDS(static_cast<int64_t>(j) * a.run.paths + nl, save_len, kDbgBasketSave))
                        a.run.save[static_cast<int64_t>(j) * a.run.paths + nl] = c.s0[j];
            }
            NormalReader rd;
            rd.init(n, a.run.rk);
            for (int i = 0; i < M; ++i) {
                // log-Euler accumulates L z straight into the state (|y| = O(1):
                // ~65 roundings of <= 3e-8 per step, ~2e-6 rms over 252 steps);
                // Euler needs dW apart because the step is multiplicative.
                f32x2 dw[SCHEME == MC_EULER ? H : 1];
                if (SCHEME == MC_EULER) {
#pragma unroll
                    for (int q = 0; q < H; ++q) dw[q] = pack2(0.0f, 0.0f);
                } else {
#pragma unroll
                    for (int q = 0; q < H; ++q) x[q] = fadd2(x[q], pack2(c.drift[2 * q], c.drift[2 * q + 1]));
                }
                // dW = Lhat z, column by column as the normals are produced;
                // column k updates the pairs q >= k/2 with (z_k, z_k).  The
                // next block of four normals is drawn before this block's
                // products (independent work while the SFU results arrive).
                float4 znext = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (EXACT) znext = normals4(static_cast<uint64_t>(i) * (D / 4), n, a.run.rk);
#pragma unroll
                for (int kb = 0; kb < D / 4 + (D % 4 ? 1 : 0); ++kb) {
                    float zz[4];
                    if (EXACT) {
                        const float4 z4 = znext;
                        if (kb + 1 < D / 4) znext = normals4(static_cast<uint64_t>(i) * (D / 4) + kb + 1, n, a.run.rk);
                        zz[0] = z4.x; zz[1] = z4.y; zz[2] = z4.z; zz[3] = z4.w;
                    } else {
#pragma unroll
                        for (int l = 0; l < 4; ++l) {
                            const int k = 4 * kb + l;
                            zz[l] = (k < D && k < d) ? rd.get(static_cast<uint64_t>(i) * d + k) : 0.0f;
                        }
                    }
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int k = 4 * kb + l;
                        if (k < D) {
                            const f32x2 z2 = pack2(zz[l], zz[l]);
#pragma unroll
                            for (int q = k / 2; q < H; ++q) {
                                const f32x2 Lq = c.Lp[basket_pair_base(D, k) + q - k / 2];
                                if (SCHEME == MC_EULER) dw[q] = ffma2(Lq, z2, dw[q]);
                                else x[q] = ffma2(Lq, z2, x[q]);
                            }
                        }
                    }
                    if (!SAVE) __syncthreads();
                }
                if (SCHEME == MC_EULER) {
#pragma unroll
                    for (int q = 0; q < H; ++q)
                        x[q] = ffma2(x[q], fadd2(pack2(c.drift[2 * q], c.drift[2 * q + 1]), dw[q]), x[q]);
                }
                if (STATS && !SAVE && SCHEME == MC_LOG_EULER) {
                    // monitored basket: sum of (w_a S0_a) 2^{x_a}, asset pairs
                    static_assert(D % 2 == 0 && (sizeof(unsigned long long) * basket_pair_count(D) + sizeof(float) * D) % 8 == 0,
                                  "ws0 is read as 8-byte pairs");
                    f32x2 u2 = pack2(0.0f, 0.0f);
#pragma unroll
                    for (int q = 0; q < H; ++q)
                        u2 = ffma2(reinterpret_cast<const f32x2 *>(c.ws0)[q],
                                   pack2(ex2_approx(lo_of(x[q])), ex2_approx(hi_of(x[q]))), u2);
                    st.add(lo_of(u2) + hi_of(u2));
                } else if (STATS || (SAVE && ((i + 1) % a.run.save_every) == 0)) {
                    float u = 0.0f;
                    const int64_t slot = (i + 1) / a.run.save_every;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const float xj = elem(x, j);
                        const float Sj = (SCHEME == MC_LOG_EULER) ? c.s0[j] * ex2_approx(xj) : xj;
                        if (STATS) u = fmaf(c.w[j], Sj, u);
                        if (SAVE && ((i + 1) % a.run.save_every) == 0 && j < d &&
                            GBMC_IN_BOUNDS((slot * d + j) * a.run.paths + nl, save_len, kDbgBasketSave))
                            a.run.save[(slot * d + j) * a.run.paths + nl] = Sj;
                    }
                    if (STATS) st.add(u);
                }
            }
            float u = 0.0f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (SCHEME == MC_LOG_EULER) u = fmaf(c.ws0[j], ex2_approx(elem(x, j)), u);
                else u = fmaf(c.w[j], elem(x, j), u);
            }
            uT = u;
            avg = st.sum * inv_m;
        }
        if (a.pay.n > 0) accumulate_payoffs(s_acc, a.pay, valid, uT, avg, st);
    }
    if (a.pay.n > 0) block_finish(s_acc, s_red, a.pay.n, a.red);
}

template <int D, int SCHEME, bool STATS, bool SAVE, bool EXACT>
const void *basket_fn()
{
    return reinterpret_cast<const void *>(&basket_fp32_kernel<D, SCHEME, STATS, SAVE, EXACT>);
}

template <int D, int SCHEME>
const void *basket_select_impl(const BasketArgs &a)
{
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    const bool save = a.run.save != nullptr;
    const bool exact = (a.d == D) && (D % 4 == 0);
    if (save) return basket_fn<D, SCHEME, false, true, false>();
    if (stats) return exact ? basket_fn<D, SCHEME, true, false, true>() : basket_fn<D, SCHEME, true, false, false>();
    return exact ? basket_fn<D, SCHEME, false, false, true>() : basket_fn<D, SCHEME, false, false, false>();
}

}  // namespace basket_detail

template <int D, int SCHEME>
const void *basket_select_scheme(const BasketArgs &a)
{
    return basket_detail::basket_select_impl<D, SCHEME>(a);
}

#define GBMC_INSTANTIATE_BASKET(D, SCHEME) \
    template const void *basket_select_scheme<D, SCHEME>(const BasketArgs &a);
#endif  // GBMC_BASKET_IMPL

}  // namespace gbmc
