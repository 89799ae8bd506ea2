// Portfolio risk (Sec. VI.B: VaR and CVaR of a portfolio of options on
// correlated underlyings) and the Monte Carlo labels of its pricing
// surrogate.  Kernels:
//   label_kernel     one parameter point (S/K, sigma, tau, r, K/H) per CTA:
//                    Monte Carlo price / K of a call, up-and-out when K/H > 0
//                    (daily monitoring), the training labels of the network;
//   outer_kernel     one risk scenario per thread: correlated one-period GBM
//                    move of every underlying over the horizon h;
//   nested_kernel    one (scenario, underlying) per CTA: inner Monte Carlo
//                    revaluation of that underlying's options at the scenario
//                    state (the yardstick of the surrogate, and its fallback);
//   features_kernel  network inputs of every (scenario, option) pair;
//   pnl_kernel       one scenario per CTA: portfolio PnL from the revalued
//                    options (FP64 sum over options);
//   tail_kernel      one CTA: bitonic sort of the losses, VaR and CVaR.
// Random streams: the stream index carries a domain tag in its top byte
// (2 outer scenarios, 3 inner paths, 4 labels, 5 base values) so that the
// domains never share normals.
#include <cmath>

#include "mc_kernels.cuh"
#include "risk.cuh"

namespace gbmc {
namespace {

__device__ __forceinline__ uint64_t tag(uint64_t domain, uint64_t idx) { return (domain << 56) | idx; }

// Network inputs from the raw point (S/K, sigma, tau, r, K/H): each mapped
// from its parameter-box range to about [-1, 1] (the constants of mc.h).
__device__ __forceinline__ void surrogate_inputs(float sk, float sig, float tau, float r, float kh, float *f)
{
    f[0] = (sk - 1.05f) * (1.0f / 0.55f);
    f[1] = (sig - 0.25f) * (1.0f / 0.15f);
    f[2] = tau - 1.0f;
    f[3] = (r - 0.04f) * (1.0f / 0.04f);
    f[4] = (kh - 0.45f) * (1.0f / 0.45f);
}

// ------------------------------ labels -----------------------------------
// GREEKS: also the pathwise sensitivities of each European point's label
// (Sec. I.A.3), per path 1{S_T > 1} S_T / S (d/d S/K) and
// 1{S_T > 1} S_T (sqrt(dt) sum z - sigma tau) (d/d sigma), discounted and
// averaged like the label; barrier points (a knock indicator has no pathwise
// derivative) get NaN.
template <bool GREEKS>
__global__ void __launch_bounds__(256) label_kernel(int64_t npts, const float *__restrict__ pts, int paths,
                                                    float steps_per_year, const __grid_constant__ RoundKeys rk,
                                                    float *__restrict__ labels, float *__restrict__ inputs,
                                                    float *__restrict__ dlabels)
{
    __shared__ double s_red[3][8];
    for (int64_t p = blockIdx.x; p < npts; p += gridDim.x) {
        const float sk = pts[p * 5 + 0], sig = pts[p * 5 + 1], tau = pts[p * 5 + 2], r = pts[p * 5 + 3],
                    kh = pts[p * 5 + 4];
        if (inputs && threadIdx.x == 0) surrogate_inputs(sk, sig, tau, r, kh, inputs + p * 5);
        const int M = max(1, __float2int_rn(tau * steps_per_year));
        const float dt = tau / M;
        const float H = kh > 0.0f ? 1.0f / kh : INFINITY;  // barrier in units of K
        const float a = kLog2e * (r - 0.5f * sig * sig) * dt, b = kLog2e * sig * sqrtf(dt);
        const bool greeks = GREEKS && !(kh > 0.0f);
        float acc = 0.0f, accd = 0.0f, accv = 0.0f;
        if (!(sk >= H)) {  // already at or above the barrier on the current date: worthless
            for (int path = threadIdx.x; path < paths; path += blockDim.x) {
                const uint64_t n = tag(4, (static_cast<uint64_t>(p) << 16) | static_cast<uint64_t>(path));
                float y = 0.0f, zs = 0.0f;
                bool alive = true;
                for (int q = 0; q < (M + 3) / 4; ++q) {
                    const float4 z = normals4(static_cast<uint64_t>(q), n, rk);
                    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        if (4 * q + l < M) {
                            y += fmaf(b, zz[l], a);
                            if (GREEKS) zs += zz[l];
                            if (sk * ex2_approx(y) >= H) alive = false;
                        }
                    }
                }
                const float g = ex2_approx(y), ST = sk * g;
                acc += alive ? fmaxf(ST - 1.0f, 0.0f) : 0.0f;
                if (greeks && ST > 1.0f) {
                    accd += g;
                    accv += ST * fmaf(sqrtf(dt), zs, -sig * tau);
                }
            }
        }
        const double v[3] = {warp_sum_d(static_cast<double>(acc)), GREEKS ? warp_sum_d(static_cast<double>(accd)) : 0.0,
                             GREEKS ? warp_sum_d(static_cast<double>(accv)) : 0.0};
        if ((threadIdx.x & 31) == 0)
            for (int k = 0; k < (GREEKS ? 3 : 1); ++k) s_red[k][threadIdx.x >> 5] = v[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < (GREEKS ? 3 : 1); ++k)
                for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t[k] += s_red[k][w];
            const double disc = exp(-static_cast<double>(r) * tau) / paths;
            if (GBMC_IN_BOUNDS(p, npts, kDbgLabelOut)) labels[p] = static_cast<float>(disc * t[0]);
            if (GREEKS) {
                dlabels[2 * p] = greeks ? static_cast<float>(disc * t[1]) : __int_as_float(0x7fc00000);
                dlabels[2 * p + 1] = greeks ? static_cast<float>(disc * t[2]) : __int_as_float(0x7fc00000);
            }
        }
        __syncthreads();
    }
}

// ------------------------------ scenarios --------------------------------
// Lc: [d x d] FP32 of sqrt(h) diag(sigma) Lrho (lower); drift_u = (mu - sigma^2/2) h.
__global__ void outer_kernel(int64_t nscen, int64_t off, int d, const float *__restrict__ Lc,
                             const float *__restrict__ drift, const float *__restrict__ s0, const __grid_constant__ RoundKeys rk,
                             float *__restrict__ Sp)
{
    extern __shared__ float sL[];
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) sL[i] = Lc[i];
    __syncthreads();
    float z[kRiskMaxUnder];
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < nscen;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        NormalReader rd;
        rd.init(tag(2, static_cast<uint64_t>(off + s)), rk);  // global scenario index
        for (int u = 0; u < d; ++u) z[u] = rd.get(u);
        for (int u = 0; u < d; ++u) {
            float w = 0.0f;
            for (int k = 0; k <= u; ++k) w = fmaf(sL[u * d + k], z[k], w);
            Sp[s * d + u] = s0[u] * expf(drift[u] + w);
        }
    }
}

// ------------------------------ nested -----------------------------------
// One CTA per (scenario s, underlying u); inner paths from S'_u, daily steps,
// every option of u valued at its remaining maturity; out[s*d + u] =
// sum_{o of u} pos_o (V_o(s) - base_o) in FP64.
__global__ void __launch_bounds__(256) nested_kernel(const __grid_constant__ RiskArgs a, const float *__restrict__ Sp, double *__restrict__ out)
{
    __shared__ double s_v[kRiskMaxOptPerUnder];
    __shared__ double s_red[8][kRiskMaxOptPerUnder];
    const int d = a.d;
    const int64_t pair = blockIdx.x;
    const int64_t s = pair / d;
    const int u = static_cast<int>(pair % d);
    const int o0 = a.under_start[u], no = a.under_start[u + 1] - o0;  // options of u, sorted by maturity
    const int hs = Sp ? 0 : a.horizon_steps;  // base date: full maturity
    const float S1 = Sp ? Sp[s * d + u] : a.s0[u];
    const float sig = a.sigma[u];
    const float dt = a.dt;
    const float aa = kLog2e * (a.r - 0.5f * sig * sig) * dt, bb = kLog2e * sig * sqrtf(dt);
    const int maxrem = no > 0 ? a.rem[o0 + no - 1] + hs : 0;
    float acc[kRiskMaxOptPerUnder];
#pragma unroll
    for (int j = 0; j < kRiskMaxOptPerUnder; ++j) acc[j] = 0.0f;
    const uint64_t gpair = static_cast<uint64_t>(a.scen_off + s) * d + u;  // global (scenario, underlying)
    const uint64_t base_idx = Sp ? (gpair << 16) : (static_cast<uint64_t>(u) << 24);
    const uint64_t domain = Sp ? 3 : 5;
    for (int path = threadIdx.x; path < a.inner; path += blockDim.x) {
        const uint64_t n = tag(domain, base_idx | static_cast<uint64_t>(path));
        float y = 0.0f, mx = -INFINITY;  // log2(S/S1) and its running maximum over the dates
        int jn = 0;                      // next option to mature
        for (int q = 0; q < (maxrem + 3) / 4; ++q) {
            const float4 z = normals4(static_cast<uint64_t>(q), n, a.rk);
            const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int step = 4 * q + l + 1;
                if (step <= maxrem) {
                    y += fmaf(bb, zz[l], aa);
                    mx = fmaxf(mx, y);
                    while (jn < no && a.rem[o0 + jn] + hs == step) {
                        const int o = o0 + jn;
                        const float ST = S1 * ex2_approx(y);
                        const float K = a.strike[o];
                        float f = a.kind[o] == MC_PUT ? fmaxf(K - ST, 0.0f) : fmaxf(ST - K, 0.0f);
                        if (a.kind[o] == MC_UO_CALL && S1 * ex2_approx(mx) >= a.barrier[o]) f = 0.0f;
                        acc[jn] += f;
                        ++jn;
                    }
                }
            }
        }
    }
    // block reduction per option (FP64)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < no; ++j) {
        const double v = warp_sum_d(static_cast<double>(acc[j]));
        if (lane == 0) s_red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < no) {
        const int j = threadIdx.x, o = o0 + j;
        double t = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w][j];
        double V = exp(-static_cast<double>(a.r) * (a.rem[o] + hs) * dt) * t / a.inner;
        if (a.kind[o] == MC_UO_CALL && S1 >= a.barrier[o]) V = 0.0;  // knocked out on the current date
        s_v[j] = V;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < no; ++j) {
            const int o = o0 + j;
            if (Sp) t += a.pos[o] * (s_v[j] - a.base[o]);
            else a.base_out[o] = s_v[j];
        }
        if (Sp) out[pair] = t;
    }
}

// ------------------------------ surrogate --------------------------------
// x[(s * nopt + o) * 5 ..]: network inputs of S/K, sigma, tau_remaining, r, K/H (0 = no barrier);
// Sp == nullptr: the base date (S0, full maturity).
__global__ void features_kernel(RiskArgs a, int64_t nscen, const float *__restrict__ Sp, float *__restrict__ x)
{
    const int64_t total = nscen * a.nopt;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t s = i / a.nopt;
        const int o = static_cast<int>(i % a.nopt);
        const int u = a.under[o];
        const float S = Sp ? Sp[s * a.d + u] : a.s0[u];
        const float K = a.strike[o];
        const int steps = Sp ? a.rem[o] : a.rem[o] + a.horizon_steps;
        surrogate_inputs(S / K, a.sigma[u], steps * a.dt, a.r, a.kind[o] == MC_UO_CALL ? K / a.barrier[o] : 0.0f,
                         x + i * 5);
    }
}

// Value of option o from the network output y = V_call / K at its features.
__device__ __forceinline__ double option_value(const RiskArgs &a, int o, float S, float y, int steps)
{
    const double K = a.strike[o];
    double call = K * static_cast<double>(y);
    if (a.kind[o] == MC_UO_CALL) {
        if (S >= a.barrier[o]) return 0.0;
        return fmax(call, 0.0);
    }
    if (a.kind[o] == MC_PUT) return call - S + K * exp(-static_cast<double>(a.r) * steps * a.dt);  // parity
    return call;
}

// base_out[o] (Sp == nullptr) or pnl[s] = sum_o pos_o (V_o(s) - base_o).
__global__ void __launch_bounds__(256) pnl_kernel(RiskArgs a, const float *__restrict__ Sp, const float *__restrict__ y,
                                                  double *__restrict__ pnl)
{
    __shared__ double s_red[8];
    const int64_t s = blockIdx.x;
    double t = 0.0;
    for (int o = threadIdx.x; o < a.nopt; o += blockDim.x) {
        const int u = a.under[o];
        const float S = Sp ? Sp[s * a.d + u] : a.s0[u];
        const int steps = Sp ? a.rem[o] : a.rem[o] + a.horizon_steps;
        const double V = option_value(a, o, S, y[s * a.nopt + o], steps);
        if (Sp) t += a.pos[o] * (V - a.base[o]);
        else a.base_out[o] = V;
    }
    if (!Sp) return;
    t = warp_sum_d(t);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) v += s_red[w];
        pnl[s] = v;
    }
}

// pnl[s] = sum_u contrib[s*d + u] (nested path).
__global__ void sum_under_kernel(int64_t nscen, int d, const double *contrib, double *pnl)
{
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < nscen;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double t = 0.0;
        for (int u = 0; u < d; ++u) t += contrib[s * d + u];
        pnl[s] = t;
    }
}

// ------------------------------ VaR / CVaR -------------------------------
// One CTA of 1024 threads: losses l = -pnl padded to a power of two with
// -inf, bitonic sort descending in global memory (work), then
// VaR = the k-th largest loss, k = ceil((1 - alpha) n), and CVaR = the mean of
// the losses strictly above VaR (VaR itself if there is none).
__global__ void __launch_bounds__(1024) tail_kernel(int64_t n, const double *pnl, double *work, int64_t npow2,
                                                    double alpha, double *res)
{
    for (int64_t i = threadIdx.x; i < npow2; i += blockDim.x) work[i] = i < n ? -pnl[i] : -INFINITY;
    __syncthreads();
    for (int64_t k = 2; k <= npow2; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const bool desc = (i & k) == 0;
                    const double x = work[i], y = work[l];
                    if (desc ? (x < y) : (x > y)) {
                        work[i] = y;
                        work[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    __shared__ double s_red[32];
    int64_t kk = static_cast<int64_t>(ceil((1.0 - alpha) * static_cast<double>(n) - 1e-9));
    if (kk < 1) kk = 1;
    const double var = work[kk - 1];
    double t = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < kk; i += blockDim.x) {
        if (work[i] > var) { t += work[i]; c += 1.0; }
    }
    t = warp_sum_d(t);
    c = warp_sum_d(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_red[warp] = t; }
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 32; ++w) tot += s_red[w];
    __syncthreads();
    if (lane == 0) s_red[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double cnt = 0.0;
        for (int w = 0; w < 32; ++w) cnt += s_red[w];
        res[0] = var;
        res[1] = cnt > 0.0 ? tot / cnt : var;
        res[2] = cnt;
    }
}

}  // namespace

cudaError_t launch_labels(int64_t npts, const float *pts, int paths, float spy, const RoundKeys &rk,
                          float *labels, float *inputs, float *dlabels, cudaStream_t s)
{
    const int64_t g = npts < 1216 * 4 ? npts : 1216 * 4;
    if (dlabels)
        label_kernel<true><<<static_cast<int>(g), 256, 0, s>>>(npts, pts, paths, spy, rk, labels, inputs, dlabels);
    else
        label_kernel<false><<<static_cast<int>(g), 256, 0, s>>>(npts, pts, paths, spy, rk, labels, inputs, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_outer(int64_t nscen, int64_t off, int d, const float *Lc, const float *drift, const float *s0,
                         const RoundKeys &rk, float *Sp, cudaStream_t s)
{
    const int64_t g = (nscen + 127) / 128;
    outer_kernel<<<static_cast<int>(g < 4096 ? g : 4096), 128, d * d * sizeof(float), s>>>(nscen, off, d, Lc, drift,
                                                                                            s0, rk, Sp);
    return cudaGetLastError();
}

cudaError_t launch_nested(const RiskArgs &a, int64_t nscen, const float *Sp, double *contrib, cudaStream_t s)
{
    const int64_t g = Sp ? nscen * a.d : a.d;
    nested_kernel<<<static_cast<int>(g), 256, 0, s>>>(a, Sp, contrib);
    return cudaGetLastError();
}

cudaError_t launch_sum_under(int64_t nscen, int d, const double *contrib, double *pnl, cudaStream_t s)
{
    const int64_t g = (nscen + 255) / 256;
    sum_under_kernel<<<static_cast<int>(g < 4096 ? g : 4096), 256, 0, s>>>(nscen, d, contrib, pnl);
    return cudaGetLastError();
}

cudaError_t launch_features(const RiskArgs &a, int64_t nscen, const float *Sp, float *x, cudaStream_t s)
{
    features_kernel<<<4096, 256, 0, s>>>(a, nscen, Sp, x);
    return cudaGetLastError();
}

cudaError_t launch_pnl(const RiskArgs &a, int64_t nscen, const float *Sp, const float *y, double *pnl, cudaStream_t s)
{
    pnl_kernel<<<static_cast<int>(Sp ? nscen : 1), 256, 0, s>>>(a, Sp, y, pnl);
    return cudaGetLastError();
}

cudaError_t launch_tail(int64_t n, const double *pnl, double *work, int64_t npow2, double alpha, double *res,
                        cudaStream_t s)
{
    tail_kernel<<<1, 1024, 0, s>>>(n, pnl, work, npow2, alpha, res);
    return cudaGetLastError();
}

}  // namespace gbmc
