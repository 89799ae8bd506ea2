// Factor-model correlated GBM basket (the correlation of the synthetic
// markets is a k-factor model, rho = B B^T + diag(e^2)): per step the path
// draws k common normals z and d idiosyncratic normals eps and moves
//   log2(S_a / S0_a) += drift_a + e'_a eps_a + sum_j B'_ja z_j
// (log-Euler; Euler: S_a <- S_a (1 + r dt + dW_a)), with B'_ja = c sqrt(dt)
// sigma_a B_aj and e'_a = c sqrt(dt) sigma_a e_a: O(d k) work per step
// instead of the O(d^2) Cholesky contraction, exact in law (Sec. II.A.2's
// Euler step with sigma(X) = diag(X) diag(sigma) [B | diag(e)]).
//   * a warp carries 4 paths; each lane owns 8 assets of each, so a group
//     of G = ceil(d / 256) warps carries 4 paths of up to 256 G assets;
//   * lanes 0 .. k - 1 draw the 4 paths' common normals (one Philox block
//     each) and broadcast them by shuffles; every lane draws the
//     idiosyncratic normals of its 8 assets;
//   * B' is staged in shared memory as [factor][asset], so one 16-byte load
//     feeds 16 FMAs (4 assets x 4 paths);
//   * GREEKS (log-Euler, one European call or put): at T each lane adds its
//     assets' pathwise delta and vega terms of its 4 paths (Sec. I.A.3; the
//     normals held fixed, ln S_a = ln S0_a + (r - sigma_a^2/2) T + sigma_a X_a)
//     to per-CTA sums in shared memory, and the path holders add rho's.
// Stream layout: normals i (k + d) + j (z_j) and i (k + d) + k + a (eps_a).
#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kP = 4;   // paths per warp
constexpr int kA = 8;   // assets per lane

template <int SCHEME, bool STATS, bool EXACT, bool GREEKS>
__global__ void __launch_bounds__(kBlock, 2) factor_kernel(const __grid_constant__ FactorArgs a)
{
    extern __shared__ float smem[];
    const int d = a.d, k = a.k, G = a.G, dp = 256 * G;
    float *sB = smem;                 // [k][dp]
    float *sE = sB + k * dp;          // e'
    float *sDr = sE + dp;             // drift
    float *sWs = sDr + dp;            // w S0 (log-Euler U) or w (Euler U)
    float *sPart = sWs + dp;          // [kWarps][kP] partial U of each warp
    float *sG = sPart + kWarps * kP;  // GREEKS: [2d + 1][2] sums of the terms and their squares
    __shared__ AccSlot s_acc[kWarps * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int i = t; i < k * dp; i += kBlock) sB[i] = a.Bp[i];
    for (int i = t; i < dp; i += kBlock) {
        sE[i] = a.ep[i];
        sDr[i] = a.drift[i];
        sWs[i] = SCHEME == MC_LOG_EULER ? a.ws0[i] : a.w[i];
    }
    for (int i = t; i < kWarps * a.pay.n * 2; i += kBlock) s_acc[i] = 0.0f;
    if (GREEKS)
        for (int i = t; i < (2 * d + 1) * 2; i += kBlock) sG[i] = 0.0f;
    __syncthreads();

    const int group = warp / G, gw = warp % G, groups = kWarps / G;
    const int a0 = 256 * gw + kA * lane;  // first asset of this lane
    const int per_cta = kP * groups;
    const int64_t ntiles = (a.run.paths + per_cta - 1) / per_cta;
    const int M = a.run.steps, stride = k + d, nzb = k / 4;
    const float inv_m = 1.0f / static_cast<float>(M);

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t n[kP];
        bool valid[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            const int64_t pl = tile * per_cta + kP * group + p;
            valid[p] = pl < a.run.paths;
            n[p] = static_cast<uint64_t>(a.run.path_offset + (valid[p] ? pl : 0));
        }
        float x[kP][kA];
#pragma unroll
        for (int p = 0; p < kP; ++p)
#pragma unroll
            for (int e = 0; e < kA; ++e) x[p][e] = SCHEME == MC_LOG_EULER ? 0.0f : a.s0[a0 + e];
        float sum = 0.0f, umax = -INFINITY, umin = INFINITY, uT = 0.0f;  // lanes 0..3 of warp gw = 0: path `lane`
        NormalReader rd[kP];
        if (!EXACT) {
#pragma unroll
            for (int p = 0; p < kP; ++p) rd[p].init(n[p], a.run.rk);
        }
        for (int i = 0; i < M; ++i) {
            const uint64_t base = static_cast<uint64_t>(i) * stride;
            // common factors: z[p][j]
            float z[kP][kFactorMax];
            if (EXACT) {
                float4 zb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (lane < kP * nzb) {
                    const int p = lane / nzb, b = lane % nzb;
                    uint64_t np = n[0];
#pragma unroll
                    for (int q = 1; q < kP; ++q) np = (p == q) ? n[q] : np;
                    zb = normals4(base / 4 + b, np, a.run.rk);
                }
#pragma unroll
                for (int p = 0; p < kP; ++p)
#pragma unroll
                    for (int j = 0; j < kFactorMax; ++j) {
                        const int src = p * nzb + (j >> 2);
                        const float c = (j & 3) == 0 ? zb.x : (j & 3) == 1 ? zb.y : (j & 3) == 2 ? zb.z : zb.w;
                        const float v = __shfl_sync(0xffffffffu, c, src < 32 ? src : 0);
                        z[p][j] = j < k ? v : 0.0f;
                    }
            } else {
#pragma unroll
                for (int p = 0; p < kP; ++p)
#pragma unroll
                    for (int j = 0; j < kFactorMax; ++j) z[p][j] = j < k ? rd[p].get(base + j) : 0.0f;
            }
            // idiosyncratic normals and the step
            float acc[SCHEME == MC_EULER ? kP : 1][kA];
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                float eps[kA];
                if (EXACT) {
                    const uint64_t q = (base + k + a0) / 4;
                    const float4 e0 = a0 < d ? normals4(q, n[p], a.run.rk) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 e1 = a0 + 4 < d ? normals4(q + 1, n[p], a.run.rk) : make_float4(0.f, 0.f, 0.f, 0.f);
                    eps[0] = e0.x; eps[1] = e0.y; eps[2] = e0.z; eps[3] = e0.w;
                    eps[4] = e1.x; eps[5] = e1.y; eps[6] = e1.z; eps[7] = e1.w;
                } else {
#pragma unroll
                    for (int e = 0; e < kA; ++e) eps[e] = a0 + e < d ? rd[p].get(base + k + a0 + e) : 0.0f;
                }
#pragma unroll
                for (int e = 0; e < kA; ++e) {
                    const float v = fmaf(sE[a0 + e], eps[e], sDr[a0 + e]);
                    if (SCHEME == MC_LOG_EULER) x[p][e] += v;
                    else acc[p][e] = v;
                }
            }
#pragma unroll
            for (int j = 0; j < kFactorMax; ++j) {
                if (j < k) {
                    const float4 b0 = *reinterpret_cast<const float4 *>(sB + j * dp + a0);
                    const float4 b1 = *reinterpret_cast<const float4 *>(sB + j * dp + a0 + 4);
                    const float bj[kA] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int p = 0; p < kP; ++p)
#pragma unroll
                        for (int e = 0; e < kA; ++e) {
                            if (SCHEME == MC_LOG_EULER) x[p][e] = fmaf(bj[e], z[p][j], x[p][e]);
                            else acc[p][e] = fmaf(bj[e], z[p][j], acc[p][e]);
                        }
                }
            }
            if (SCHEME == MC_EULER) {
#pragma unroll
                for (int p = 0; p < kP; ++p)
#pragma unroll
                    for (int e = 0; e < kA; ++e) x[p][e] = fmaf(x[p][e], acc[p][e], x[p][e]);
            }
            if (STATS || i == M - 1) {
                // U of each path: lane partials -> warp sums -> the group's G warps
#pragma unroll
                for (int p = 0; p < kP; ++p) {
                    float u = 0.0f;
#pragma unroll
                    for (int e = 0; e < kA; ++e) {
                        const float S = SCHEME == MC_LOG_EULER ? ex2_approx(x[p][e]) : x[p][e];
                        u = a0 + e < d ? fmaf(sWs[a0 + e], S, u) : u;
                    }
                    u = warp_sum(u);
                    if (lane == 0) sPart[warp * kP + p] = u;
                }
                __syncthreads();
                if (gw == 0 && lane < kP) {
                    float u = 0.0f;
                    for (int g = 0; g < G; ++g) u += sPart[(warp + g) * kP + lane];
                    if (STATS) {
                        sum += u;
                        umax = fmaxf(umax, u);
                        umin = fminf(umin, u);
                    }
                    if (i == M - 1) uT = u;
                }
                __syncthreads();  // the partials are read before the next step writes them
            }
        }
        // payoffs: lane p (< 4) of the group's first warp holds path p
        const bool holder = gw == 0 && lane < kP;
        bool ok = false;
#pragma unroll
        for (int p = 0; p < kP; ++p) ok = (lane == p) ? valid[p] : ok;
        if (GREEKS) {
            // the payoff slope of each path to every lane of its group (the
            // partial sums are free after the last step's barrier)
            const float K = a.pay.strike[0];
            const bool put = a.pay.kind[0] == MC_PUT;
            if (holder) sPart[group * kP + lane] = ok ? (put ? (uT < K ? -1.0f : 0.0f) : (uT > K ? 1.0f : 0.0f)) : 0.0f;
            __syncthreads();
            float gp[kP];
#pragma unroll
            for (int p = 0; p < kP; ++p) gp[p] = sPart[group * kP + p];
            const float rT = a.r * a.T;
#pragma unroll
            for (int e = 0; e < kA; ++e) {
                const int col = a0 + e;
                if (col < d) {
                    const float wa = a.w[col], s0a = a.s0[col], sga = a.sigma[col];
                    const float c = fmaf(0.5f * sga * sga, a.T, rT);  // (r + sigma^2 / 2) T
                    float d1 = 0.0f, d2 = 0.0f, v1 = 0.0f, v2 = 0.0f;
#pragma unroll
                    for (int p = 0; p < kP; ++p) {
                        const float dl = gp[p] * wa * ex2_approx(x[p][e]);  // f' w_a S_a / S0_a
                        const float vg = dl * s0a * (fmaf(x[p][e], 0.6931471805599453f, -c) / sga);
                        d1 += dl;
                        d2 += dl * dl;
                        v1 += vg;
                        v2 += vg * vg;
                    }
                    if (d1 != 0.0f || d2 != 0.0f) {
                        atomicAdd(&sG[2 * col], d1);
                        atomicAdd(&sG[2 * col + 1], d2);
                        atomicAdd(&sG[2 * (d + col)], v1);
                        atomicAdd(&sG[2 * (d + col) + 1], v2);
                    }
                }
            }
            if (holder && ok) {
                const float g = sPart[group * kP + lane];
                const float f = payoff_eval(a.pay.kind[0], K, INFINITY, uT, 0.0f, 0.0f, 0.0f);
                const float rr = g * uT * a.T - a.T * f;
                atomicAdd(&sG[4 * d], rr);
                atomicAdd(&sG[4 * d + 1], rr * rr);
            }
            __syncthreads();  // the slopes are read before the next tile's last step rewrites them
        }
        for (int pi = 0; pi < a.pay.n; ++pi) {
            const float f = (holder && ok) ? payoff_eval(a.pay.kind[pi], a.pay.strike[pi], a.pay.barrier[pi], uT,
                                                         sum * inv_m, umax, umin)
                                           : 0.0f;
            warp_accumulate(s_acc, a.pay.n, pi, f);
        }
    }
    if (GREEKS) {
        __syncthreads();
        float *dst = a.gpart + static_cast<size_t>(blockIdx.x) * (2 * d + 1) * 2;
        for (int i = t; i < (2 * d + 1) * 2; i += kBlock) dst[i] = sG[i];
    }
    block_finish(s_acc, s_red, a.pay.n, a.red);
}

// out[g] = disc (mean, standard error) of Greek g from the CTAs' sums.
__global__ void factor_greeks_finish_kernel(int nv, int grid, const float *__restrict__ gpart, int64_t paths,
                                            double disc, mc_result *__restrict__ out)
{
    const double N = static_cast<double>(paths);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nv; g += gridDim.x * blockDim.x) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < grid; ++b) {
            s1 += static_cast<double>(gpart[(static_cast<size_t>(b) * nv + g) * 2]);
            s2 += static_cast<double>(gpart[(static_cast<size_t>(b) * nv + g) * 2 + 1]);
        }
        const double mean = s1 / N, var = fmax(s2 / N - mean * mean, 0.0);
        mc_result r;
        r.price = disc * mean;
        r.se = paths > 1 ? disc * sqrt(var / (N - 1.0)) : 0.0;
        out[g] = r;
    }
}

template <int SCHEME, bool STATS, bool EXACT, bool GREEKS = false>
const void *fn() { return reinterpret_cast<const void *>(&factor_kernel<SCHEME, STATS, EXACT, GREEKS>); }

template <int SCHEME, bool STATS>
const void *pick(const FactorArgs &a) { return a.exact4 ? fn<SCHEME, STATS, true>() : fn<SCHEME, STATS, false>(); }

const void *select(const FactorArgs &a)
{
    if (a.greeks)  // log-Euler, European payoff (checked by the caller)
        return a.exact4 ? fn<MC_LOG_EULER, false, true, true>() : fn<MC_LOG_EULER, false, false, true>();
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    if (a.scheme == MC_LOG_EULER) return stats ? pick<MC_LOG_EULER, true>(a) : pick<MC_LOG_EULER, false>(a);
    return stats ? pick<MC_EULER, true>(a) : pick<MC_EULER, false>(a);
}

}  // namespace

size_t factor_smem_bytes(const FactorArgs &a)
{
    const int dp = 256 * a.G;
    return static_cast<size_t>(a.k * dp + 3 * dp + kWarps * kP + (a.greeks ? (2 * a.d + 1) * 2 : 0)) * sizeof(float);
}

cudaError_t launch_factor_greeks_finish(const FactorArgs &a, int grid, double disc, mc_result *out, cudaStream_t s)
{
    const int nv = 2 * a.d + 1;
    factor_greeks_finish_kernel<<<(nv + 255) / 256, 256, 0, s>>>(nv, grid, a.gpart, a.run.paths, disc, out);
    return cudaGetLastError();
}

cudaError_t launch_factor(const FactorArgs &a, int grid, cudaStream_t s)
{
    const void *f = select(a);
    const size_t smem = factor_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<FactorArgs *>(&a)};
    return cudaLaunchKernel(f, dim3(grid), dim3(kBlock), args, smem, s);
}

int factor_occupancy(const FactorArgs &a)
{
    const void *f = select(a);
    const size_t smem = factor_smem_bytes(a);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, smem) != cudaSuccess) return 0;
    return nb;
}

int factor_paths_per_cta(const FactorArgs &a) { return kP * (kWarps / a.G); }

}  // namespace gbmc
