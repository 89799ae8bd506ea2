// Pathwise correlation sensitivities of a European basket call or put
// (Sec. I.A.3: sensitivities to model parameters; Sec. VI.A.2 obtains basket
// sensitivities by differentiating the simulation), reverse mode.
//
// Log-Euler with constant coefficients: after M steps
//   x_a(T) = log S0_a + M drift_a + sqrt(dt) sigma_a (Lrho W)_a,  W = sum_i z_i,
// so the terminal prices depend on the correlation only through the sum W of
// the path's normal vectors.  The payoff's slope in x_a is
// u_a = w_a S_a(T) 1{U > K} (call), -w_a S_a(T) 1{U < K} (put), and
//   dP/dLrho[a][b] = disc sqrt(dt) sigma_a E[u_a W_b],   b <= a.
// The path kernel accumulates H = sum_paths u W^T per CTA (an FP32 outer-
// product sum over tiles of 32 paths staged in shared memory); a second
// kernel sums the CTA partials in FP64 into batches; the adjoint kernel maps
// each batch's dP/dLrho through the transpose of the Cholesky derivative,
//   S = Lrho^-T Phi(Lrho^T Lbar) Lrho^-1   (Phi: lower triangle, diagonal
//   halved),  dP/dcorr[a][b] = S_ab + S_ba  (a != b, both entries moved),
// and the last kernel forms means and batch-means standard errors.
#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kD = kCorrMaxD;     // assets (padded)
constexpr int kThreads = 128;     // paths per tile
constexpr int kQuarter = 32;      // paths staged per outer-product pass
constexpr int kStride = kD + 4;   // shared row stride (floats; 16-B aligned rows)

template <bool EXACT>
__global__ void __launch_bounds__(kThreads) corr_path_kernel(const __grid_constant__ CorrArgs a, const CorrConst c)
{
    __shared__ __align__(16) float su[kQuarter * kStride];   // w_a S_a(T) of the staged paths
    __shared__ __align__(16) float sw[kQuarter * kStride];   // W of the staged paths
    __shared__ float s_slope[kQuarter];
    __shared__ float sh[32 * kThreads];                       // this CTA's H, thread t owns column t
    __shared__ AccSlot s_acc[(kThreads / 32) * 2];
    __shared__ double s_red[32];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int j = 0; j < 32; ++j) sh[j * kThreads + t] = 0.0f;
    if (t < (kThreads / 32) * 2) s_acc[t] = 0.0f;
    __syncthreads();

    const int M = a.run.steps, d = a.d;
    const float fM = static_cast<float>(M);
    const int64_t ntiles = (a.run.paths + kThreads - 1) / kThreads;
    // H entries of this thread: row ra, columns cb .. cb + 31
    const int ra = t >> 1, cb = (t & 1) * 32;
    int64_t cnt = 0;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t nl = tile * kThreads + t;
        const bool valid = nl < a.run.paths;
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + (valid ? nl : 0));
        const int64_t left = a.run.paths - tile * kThreads;
        cnt += left < kThreads ? left : kThreads;
        float W[kD];
#pragma unroll
        for (int k = 0; k < kD; ++k) W[k] = 0.0f;
        if (EXACT) {
            const int nb = d >> 2;
            for (int i = 0; i < M; ++i) {
#pragma unroll
                for (int kb = 0; kb < kD / 4; ++kb) {
                    if (kb < nb) {
                        const float4 z = normals4(static_cast<uint64_t>(i) * nb + kb, n, a.run.rk);
                        W[4 * kb] += z.x;
                        W[4 * kb + 1] += z.y;
                        W[4 * kb + 2] += z.z;
                        W[4 * kb + 3] += z.w;
                    }
                }
            }
        } else {
            NormalReader rd;
            rd.init(n, a.run.rk);
            for (int i = 0; i < M; ++i) {
#pragma unroll
                for (int k = 0; k < kD; ++k)
                    if (k < d) W[k] += rd.get(static_cast<uint64_t>(i) * d + k);
            }
        }
        // Four passes of 32 paths (one warp each): the staging warp forms its
        // paths' terminal prices, basket and payoff; all threads then add the
        // staged paths' u W^T to their H entries.
        for (int q = 0; q < kThreads / kQuarter; ++q) {
            if (warp == q) {
                float U = 0.0f;
#pragma unroll
                for (int ra2 = 0; ra2 < kD; ++ra2) {
                    float y = fM * c.drift[ra2];
#pragma unroll
                    for (int k = 0; k <= ra2; ++k) y = fmaf(c.L[ra2 * (ra2 + 1) / 2 + k], W[k], y);
                    const float p = c.ws0[ra2] * ex2_approx(y);
                    U += p;
                    su[lane * kStride + ra2] = p;
                    sw[lane * kStride + ra2] = W[ra2];
                }
                const bool call = a.kind == MC_CALL;
                const float f = call ? fmaxf(U - a.strike, 0.0f) : fmaxf(a.strike - U, 0.0f);
                const float slope = call ? (U > a.strike ? 1.0f : 0.0f) : (U < a.strike ? -1.0f : 0.0f);
                s_slope[lane] = valid ? slope : 0.0f;
                warp_accumulate(s_acc, 1, 0, valid ? f : 0.0f);
            }
            __syncthreads();
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
            for (int p = 0; p < kQuarter; ++p) {
                const float ua = s_slope[p] * su[p * kStride + ra];
                const float4 *wr = reinterpret_cast<const float4 *>(sw + p * kStride + cb);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 w4 = wr[j];
                    acc[4 * j] = fmaf(ua, w4.x, acc[4 * j]);
                    acc[4 * j + 1] = fmaf(ua, w4.y, acc[4 * j + 1]);
                    acc[4 * j + 2] = fmaf(ua, w4.z, acc[4 * j + 2]);
                    acc[4 * j + 3] = fmaf(ua, w4.w, acc[4 * j + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) sh[j * kThreads + t] += acc[j];
            __syncthreads();
        }
    }
    float *dst = a.partials + static_cast<size_t>(blockIdx.x) * kD * kD + ra * kD + cb;
    for (int j = 0; j < 32; ++j) dst[j] = sh[j * kThreads + t];
    if (t == 0) a.counts[blockIdx.x] = static_cast<double>(cnt);
    block_finish(s_acc, s_red, 1, a.red);
}

// Batch k of B: the FP64 sum of the partials of CTAs k, k + B, k + 2B, ...
__global__ void corr_batch_kernel(const float *partials, const double *counts, int G, int B, double *Hb,
                                  double *nb)
{
    const int k = blockIdx.x;
    for (int e = threadIdx.x; e < kD * kD; e += blockDim.x) {
        double s = 0.0;
        for (int c = k; c < G; c += B) s += static_cast<double>(partials[static_cast<size_t>(c) * kD * kD + e]);
        Hb[static_cast<size_t>(k) * kD * kD + e] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int c = k; c < G; c += B) s += counts[c];
        nb[k] = s;
    }
}

// Block k < B: batch k; block B: all paths.  FP64, d <= 64, one CTA each.
// Outputs per block: dP/dLrho (lower, d-stride) and dP/dcorr (symmetric).
__global__ void __launch_bounds__(256) corr_adjoint_kernel(int d, int B, const double *Hb, const double *nb,
                                                            const double *L, const double *cfac, double *out_dl,
                                                            double *out_drho)
{
    extern __shared__ double sm[];
    double *sL = sm, *sG = sm + d * d, *sA = sm + 2 * d * d;   // Lrho, Lbar then S, A then P then X
    const int k = blockIdx.x, tid = threadIdx.x;
    double n = 0.0;
    if (k < B) n = nb[k];
    else for (int j = 0; j < B; ++j) n += nb[j];
    const double inv_n = n > 0.0 ? 1.0 / n : 0.0;
    double *odl = out_dl + static_cast<size_t>(k) * d * d, *odr = out_drho + static_cast<size_t>(k) * d * d;
    for (int e = tid; e < d * d; e += blockDim.x) {
        const int i = e / d, j = e % d;
        double h = 0.0;
        if (j <= i) {
            if (k < B) h = Hb[static_cast<size_t>(k) * kD * kD + i * kD + j];
            else for (int q = 0; q < B; ++q) h += Hb[static_cast<size_t>(q) * kD * kD + i * kD + j];
        }
        const double g = cfac[i] * h * inv_n;   // Lbar = dP/dLrho
        sG[e] = g;
        odl[e] = g;
        sL[e] = L[e];
    }
    __syncthreads();
    // A = Lrho^T Lbar, then P = Phi(A)
    for (int e = tid; e < d * d; e += blockDim.x) {
        const int i = e / d, j = e % d;
        double s = 0.0;
        if (j <= i) {
            for (int q = i; q < d; ++q) s = fma(sL[q * d + i], sG[q * d + j], s);
            if (j == i) s *= 0.5;
        }
        sA[e] = s;
    }
    __syncthreads();
    // X = P Lrho^-1 (rows, in place): x_ij = (p_ij - sum_{q > j} x_iq L_qj) / L_jj, j = i .. 0
    if (tid < d) {
        const int i = tid;
        for (int j = i; j >= 0; --j) {
            double s = sA[i * d + j];
            for (int q = j + 1; q <= i; ++q) s = fma(-sA[i * d + q], sL[q * d + j], s);
            sA[i * d + j] = s / sL[j * d + j];
        }
    }
    __syncthreads();
    // S = Lrho^-T X (columns, into sG): s_ij = (x_ij - sum_{q > i} L_qi s_qj) / L_ii, i = d-1 .. 0
    if (tid < d) {
        const int j = tid;
        for (int i = d - 1; i >= 0; --i) {
            double s = sA[i * d + j];
            for (int q = i + 1; q < d; ++q) s = fma(-sL[q * d + i], sG[q * d + j], s);
            sG[i * d + j] = s / sL[i * d + i];
        }
    }
    __syncthreads();
    for (int e = tid; e < d * d; e += blockDim.x) {
        const int i = e / d, j = e % d;
        odr[e] = (i == j) ? 0.0 : sG[i * d + j] + sG[j * d + i];
    }
}

// Mean (all-path block) and batch-means standard error
// se^2 = sum_k n_k (m_k - m)^2 / ((B - 1) N) of each output entry.
__global__ void corr_finish_kernel(int d, int B, const double *nb, const double *out_dl, const double *out_drho,
                                   mc_result *res_dl, mc_result *res_drho)
{
    const int dd = d * d;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * dd; e += gridDim.x * blockDim.x) {
        const double *o = e < dd ? out_dl : out_drho;
        const int i = e < dd ? e : e - dd;
        const double m = o[static_cast<size_t>(B) * dd + i];
        double N = 0.0, v = 0.0;
        for (int k = 0; k < B; ++k) {
            const double x = o[static_cast<size_t>(k) * dd + i] - m;
            v = fma(nb[k] * x, x, v);
            N += nb[k];
        }
        mc_result r;
        r.price = m;
        r.se = B > 1 && N > 0.0 ? sqrt(v / ((B - 1) * N)) : __longlong_as_double(0x7ff8000000000000ll);
        (e < dd ? res_dl : res_drho)[i] = r;
    }
}

// ------------------------- Asian basket (d <= 64) --------------------------
// Payoff on A = (1/M) sum_i U(t_i).  With x_a(t_i) = i drift_a + (Lhat W_i)_a
// (log2 units, W_i the sum of the first i normal vectors), the slope of the
// payoff in x_a(t_i) is u_{a,i} = f'(A) w_a S_a(t_i) / M, so
//   dP/dLrho[a][b] = disc sqrt(dt) sigma_a E[sum_i u_{a,i} W_{i,b}],
// a d x d outer product per path-step.  Per tile of 128 paths: pass 1 runs
// the paths to their averages, payoffs and slopes f'(A); pass 2 runs them
// again and, every step, stages u_i and W_i of all 128 paths in shared
// memory and adds sum_p u_p W_p^T to H (each thread an 8 x 4 block, held
// in registers across the launch).
constexpr int kAsianStride = kD + 4;  // staged row stride (floats; 16-B aligned rows)

__device__ __forceinline__ void asian_draw(bool exact, int i, int d, uint64_t n, const RoundKeys &rk,
                                           NormalReader &rd, float (&W)[kD])
{
    if (exact) {
        const int nb = d >> 2;
#pragma unroll
        for (int kb = 0; kb < kD / 4; ++kb) {
            if (kb < nb) {
                const float4 z = normals4(static_cast<uint64_t>(i) * nb + kb, n, rk);
                W[4 * kb] += z.x;
                W[4 * kb + 1] += z.y;
                W[4 * kb + 2] += z.z;
                W[4 * kb + 3] += z.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kD; ++k)
            if (k < d) W[k] += rd.get(static_cast<uint64_t>(i) * d + k);
    }
}

template <bool EXACT>
__global__ void __launch_bounds__(kThreads) corr_asian_kernel(const __grid_constant__ CorrArgs a, const CorrConst c)
{
    extern __shared__ __align__(16) float s_dyn[];
    float *sv = s_dyn;                            // [kThreads][kAsianStride] u of the staged paths
    float *sw = s_dyn + kThreads * kAsianStride;  // [kThreads][kAsianStride] W of the staged paths
    __shared__ AccSlot s_acc[(kThreads / 32) * 2];
    __shared__ double s_red[32];
    const int t = threadIdx.x;
    if (t < (kThreads / 32) * 2) s_acc[t] = 0.0f;
    __syncthreads();

    const int M = a.run.steps, d = a.d;
    const float inv_m = 1.0f / static_cast<float>(M);
    const int64_t ntiles = (a.run.paths + kThreads - 1) / kThreads;
    const int rg = t >> 4, cg = t & 15;  // H rows 8 rg .. 8 rg + 7, columns 4 cg .. 4 cg + 3
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    int64_t cnt = 0;
    const bool put = a.kind == MC_ASIAN_PUT;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t nl = tile * kThreads + t;
        const bool valid = nl < a.run.paths;
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + (valid ? nl : 0));
        const int64_t left = a.run.paths - tile * kThreads;
        cnt += left < kThreads ? left : kThreads;
        // pass 1: the average, the payoff and its slope
        float W[kD];
#pragma unroll
        for (int k = 0; k < kD; ++k) W[k] = 0.0f;
        NormalReader rd;
        rd.init(n, a.run.rk);
        float sumU = 0.0f;
        for (int i = 0; i < M; ++i) {
            asian_draw(EXACT, i, d, n, a.run.rk, rd, W);
            const float fi = static_cast<float>(i + 1);
            float U = 0.0f;
#pragma unroll
            for (int ra = 0; ra < kD; ++ra) {
                float y = fi * c.drift[ra];
#pragma unroll
                for (int k = 0; k <= ra; ++k) y = fmaf(c.L[ra * (ra + 1) / 2 + k], W[k], y);
                U = fmaf(c.ws0[ra], ex2_approx(y), U);
            }
            sumU += U;
        }
        const float A = sumU * inv_m;
        const float f = put ? fmaxf(a.strike - A, 0.0f) : fmaxf(A - a.strike, 0.0f);
        const float slope = valid ? (put ? (A < a.strike ? -1.0f : 0.0f) : (A > a.strike ? 1.0f : 0.0f)) : 0.0f;
        warp_accumulate(s_acc, 1, 0, valid ? f : 0.0f);
        // pass 2: the same paths again, u_i W_i^T of all of them every step
        const float su = slope * inv_m;
        const bool any = __syncthreads_or(su != 0.0f);  // a tile without slopes adds nothing
#pragma unroll
        for (int k = 0; k < kD; ++k) W[k] = 0.0f;
        rd.init(n, a.run.rk);
        for (int i = 0; any && i < M; ++i) {
            asian_draw(EXACT, i, d, n, a.run.rk, rd, W);
            const float fi = static_cast<float>(i + 1);
            float *vr = sv + t * kAsianStride, *wr = sw + t * kAsianStride;
#pragma unroll
            for (int ra = 0; ra < kD; ++ra) {
                float y = fi * c.drift[ra];
#pragma unroll
                for (int k = 0; k <= ra; ++k) y = fmaf(c.L[ra * (ra + 1) / 2 + k], W[k], y);
                vr[ra] = su * c.ws0[ra] * ex2_approx(y);
                wr[ra] = W[ra];
            }
            __syncthreads();
            for (int p = 0; p < kThreads; ++p) {
                const float4 v0 = *reinterpret_cast<const float4 *>(sv + p * kAsianStride + 8 * rg);
                const float4 v1 = *reinterpret_cast<const float4 *>(sv + p * kAsianStride + 8 * rg + 4);
                const float4 w4 = *reinterpret_cast<const float4 *>(sw + p * kAsianStride + 4 * cg);
                const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(vv[r], ww[q], acc[r][q]);
            }
            __syncthreads();  // the staged rows are read before the next step rewrites them
        }
    }
    float *dst = a.partials + static_cast<size_t>(blockIdx.x) * kD * kD;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[(8 * rg + r) * kD + 4 * cg + q] = acc[r][q];
    if (t == 0) a.counts[blockIdx.x] = static_cast<double>(cnt);
    block_finish(s_acc, s_red, 1, a.red);
}

size_t corr_asian_smem() { return 2 * static_cast<size_t>(kThreads) * kAsianStride * sizeof(float); }

// ------------------------- wide baskets (d > 64) ---------------------------
// Same estimator, with the per-path vectors in global memory and the two
// path-sized contractions as FP32 products:
//   W_p = sum_i z_i                        corr_wsum_kernel (chunks of 64 assets)
//   Y = W Lhat^T                           gemm_f32_abt
//   u_p,a = slope_p w_a S_a(T)             corr_u_kernel (and the price)
//   H_b = sum over batch b of u_p W_p^T     gemm_f32_atb_slices (one slice per batch)
// then dP/dLrho and the Cholesky adjoint per batch in FP64 (global memory).
constexpr int kWChunk = 64;

template <bool EXACT>
__global__ void __launch_bounds__(128) corr_wsum_kernel(const __grid_constant__ CorrArgs a, float *__restrict__ Wbuf)
{
    const int d = a.d, M = a.run.steps;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < a.run.paths; p += stride) {
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + p);
        for (int c0 = 0; c0 < d; c0 += kWChunk) {
            float W[kWChunk];
#pragma unroll
            for (int k = 0; k < kWChunk; ++k) W[k] = 0.0f;
            if (EXACT) {  // d % 4 == 0: step i's normals are blocks i d/4 .. i d/4 + d/4 - 1
                const uint64_t nb = static_cast<uint64_t>(d >> 2);
                for (int i = 0; i < M; ++i) {
#pragma unroll
                    for (int kb = 0; kb < kWChunk / 4; ++kb) {
                        if (c0 + 4 * kb < d) {
                            const float4 z = normals4(static_cast<uint64_t>(i) * nb + (c0 >> 2) + kb, n, a.run.rk);
                            W[4 * kb] += z.x;
                            W[4 * kb + 1] += z.y;
                            W[4 * kb + 2] += z.z;
                            W[4 * kb + 3] += z.w;
                        }
                    }
                }
            } else {
                NormalReader rd;
                rd.init(n, a.run.rk);
                for (int i = 0; i < M; ++i) {
#pragma unroll
                    for (int k = 0; k < kWChunk; ++k)
                        if (c0 + k < d) W[k] += rd.get(static_cast<uint64_t>(i) * d + c0 + k);
                }
            }
            float *dst = Wbuf + p * d + c0;
#pragma unroll
            for (int k = 0; k < kWChunk; ++k)
                if (c0 + k < d) dst[k] = W[k];
        }
    }
}

// One warp per path: S_a = w_a S0_a 2^{M drift_a + Y_a}, U = sum_a S_a, the
// payoff (into the price reduction) and u_a = slope S_a written over Y.
__global__ void __launch_bounds__(256) corr_u_kernel(const __grid_constant__ CorrArgs a, const float *__restrict__ drift,
                                                     const float *__restrict__ ws0, float *__restrict__ Y)
{
    __shared__ AccSlot s_acc[(256 / 32) * 2];
    __shared__ double s_red[32];
    if (threadIdx.x < (256 / 32) * 2) s_acc[threadIdx.x] = 0.0f;
    __syncthreads();
    const int d = a.d, lane = threadIdx.x & 31;
    const float fM = static_cast<float>(a.run.steps);
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const bool call = a.kind == MC_CALL;
    for (int64_t p = w0; p < a.run.paths; p += nw) {
        float *y = Y + p * d;
        float U = 0.0f;
        for (int k = lane; k < d; k += 32) {
            const float S = ws0[k] * ex2_approx(fmaf(fM, drift[k], y[k]));
            y[k] = S;
            U += S;
        }
        U = warp_sum(U);
        const float f = call ? fmaxf(U - a.strike, 0.0f) : fmaxf(a.strike - U, 0.0f);
        const float slope = call ? (U > a.strike ? 1.0f : 0.0f) : (U < a.strike ? -1.0f : 0.0f);
        for (int k = lane; k < d; k += 32) y[k] *= slope;
        warp_accumulate(s_acc, 1, 0, lane == 0 ? f : 0.0f);
    }
    block_finish(s_acc, s_red, 1, a.red);
}

// Lbar_k[q][j] = cfac_q H_k[q][j] / n_k (lower triangle) for batches k < B
// and, at k = B, for all paths (the batches' sums added in order).
__global__ void corr_lbar_kernel(int d, int B, const float *__restrict__ part, const double *__restrict__ nb,
                                 const double *__restrict__ cfac, double *__restrict__ out_dl)
{
    const int64_t dd = static_cast<int64_t>(d) * d;
    const int k = blockIdx.y;
    double n = 0.0;
    if (k < B) n = nb[k];
    else for (int j = 0; j < B; ++j) n += nb[j];
    const double inv_n = n > 0.0 ? 1.0 / n : 0.0;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < dd;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(e / d), j = static_cast<int>(e % d);
        double h = 0.0;
        if (j <= q) {
            if (k < B) h = static_cast<double>(part[k * dd + e]);
            else for (int b = 0; b < B; ++b) h += static_cast<double>(part[b * dd + e]);
        }
        out_dl[k * dd + e] = cfac[q] * h * inv_n;
    }
}

// P_k = Phi(Lrho^T Lbar_k): lower triangle, diagonal halved.
__global__ void corr_adj_a_kernel(int d, const double *__restrict__ L, const double *__restrict__ lbar,
                                  double *__restrict__ Pm)
{
    const int64_t dd = static_cast<int64_t>(d) * d;
    const int k = blockIdx.y;
    const double *G = lbar + k * dd;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < dd;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
        double s = 0.0;
        if (j <= i) {
            for (int q = i; q < d; ++q) s = fma(L[static_cast<int64_t>(q) * d + i], G[static_cast<int64_t>(q) * d + j], s);
            if (j == i) s *= 0.5;
        }
        Pm[k * dd + e] = s;
    }
}

// X_k = P_k Lrho^-1 in place, one warp per row: x_ij = (p_ij - sum_{q > j} x_iq L_qj) / L_jj,
// j = i .. 0, the sum split over the lanes.
__global__ void __launch_bounds__(256) corr_adj_x_kernel(int d, const double *__restrict__ L, double *__restrict__ Pm)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= d) return;  // whole warps
    double *X = Pm + static_cast<int64_t>(blockIdx.y) * d * d + static_cast<int64_t>(i) * d;
    for (int j = i; j >= 0; --j) {
        double s = 0.0;
        for (int q = j + 1 + lane; q <= i; q += 32) s = fma(X[q], L[static_cast<int64_t>(q) * d + j], s);
        s = warp_sum_d(s);
        if (lane == 0) X[j] = (X[j] - s) / L[static_cast<int64_t>(j) * d + j];
        __syncwarp();
    }
}

// Lt = Lrho^T (row i of Lt = column i of Lrho, contiguous for the solve below).
__global__ void corr_lt_kernel(int d, const double *__restrict__ L, double *__restrict__ Lt)
{
    const int64_t dd = static_cast<int64_t>(d) * d;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < dd;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        Lt[e] = L[(e % d) * d + e / d];
}

// S_k = Lrho^-T X_k, one thread per column (a warp's lanes on consecutive
// columns: the reads of S coalesce, those of Lt broadcast):
// s_ij = (x_ij - sum_{q > i} L_qi s_qj) / L_ii, i = d-1 .. 0, the sum in four
// independent partial sums (shorter FP64 dependency chains).
__global__ void __launch_bounds__(128) corr_adj_s_kernel(int d, const double *__restrict__ Lt,
                                                         const double *__restrict__ Pm, double *__restrict__ Sm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const int64_t off = static_cast<int64_t>(blockIdx.y) * d * d;
    const double *X = Pm + off;
    double *S = Sm + off;
    for (int i = d - 1; i >= 0; --i) {
        const double *li = Lt + static_cast<int64_t>(i) * d;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = i + 1;
        for (; q + 3 < d; q += 4) {
            s0 = fma(li[q], S[static_cast<int64_t>(q) * d + j], s0);
            s1 = fma(li[q + 1], S[static_cast<int64_t>(q + 1) * d + j], s1);
            s2 = fma(li[q + 2], S[static_cast<int64_t>(q + 2) * d + j], s2);
            s3 = fma(li[q + 3], S[static_cast<int64_t>(q + 3) * d + j], s3);
        }
        for (; q < d; ++q) s0 = fma(li[q], S[static_cast<int64_t>(q) * d + j], s0);
        S[static_cast<int64_t>(i) * d + j] = (X[static_cast<int64_t>(i) * d + j] - ((s0 + s1) + (s2 + s3))) / li[i];
    }
}

// dP/dcorr[a][b] = S_ab + S_ba (a != b), zero on the diagonal.
__global__ void corr_sym_kernel(int d, const double *__restrict__ Sm, double *__restrict__ out_drho)
{
    const int64_t dd = static_cast<int64_t>(d) * d;
    const int64_t off = static_cast<int64_t>(blockIdx.y) * dd;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < dd;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
        out_drho[off + e] = i == j ? 0.0 : Sm[off + e] + Sm[off + static_cast<int64_t>(j) * d + i];
    }
}

bool corr_asian(const CorrArgs &a) { return a.kind == MC_ASIAN_CALL || a.kind == MC_ASIAN_PUT; }

const void *corr_select(const CorrArgs &a)
{
    if (corr_asian(a))
        return a.exact4 ? reinterpret_cast<const void *>(&corr_asian_kernel<true>)
                        : reinterpret_cast<const void *>(&corr_asian_kernel<false>);
    return a.exact4 ? reinterpret_cast<const void *>(&corr_path_kernel<true>)
                    : reinterpret_cast<const void *>(&corr_path_kernel<false>);
}

size_t corr_dyn_smem(const CorrArgs &a) { return corr_asian(a) ? corr_asian_smem() : 0; }

}  // namespace

int corr_occupancy(const CorrArgs &a)
{
    const size_t smem = corr_dyn_smem(a);
    if (smem > 0 && cudaFuncSetAttribute(corr_select(a), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, corr_select(a), kThreads, smem) != cudaSuccess) return 0;
    return n;
}

int corr_block() { return kThreads; }

size_t corr_adjoint_smem(int d) { return 3 * static_cast<size_t>(d) * d * sizeof(double); }

cudaError_t launch_corr(const CorrArgs &a, const CorrConst &c, int grid, int batches, const double *L,
                        const double *cfac, double *Hb, double *nb, double *out_dl, double *out_drho,
                        mc_result *res_dl, mc_result *res_drho, cudaStream_t s)
{
    void *args[] = {const_cast<CorrArgs *>(&a), const_cast<CorrConst *>(&c)};
    const size_t dyn = corr_dyn_smem(a);
    if (dyn > 0) {
        const cudaError_t ea = cudaFuncSetAttribute(corr_select(a), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(dyn));
        if (ea != cudaSuccess) return ea;
    }
    cudaError_t e = cudaLaunchKernel(corr_select(a), dim3(grid), dim3(kThreads), args, dyn, s);
    if (e != cudaSuccess) return e;
    corr_batch_kernel<<<batches, 256, 0, s>>>(a.partials, a.counts, grid, batches, Hb, nb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = corr_adjoint_smem(a.d);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(corr_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    corr_adjoint_kernel<<<batches + 1, 256, smem, s>>>(a.d, batches, Hb, nb, L, cfac, out_dl, out_drho);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int dd2 = 2 * a.d * a.d;
    corr_finish_kernel<<<(dd2 + 255) / 256, 256, 0, s>>>(a.d, batches, nb, out_dl, out_drho, res_dl, res_drho);
    return cudaGetLastError();
}

cudaError_t launch_corr_wide(const CorrArgs &a, const CorrWide &w, int grid, cudaStream_t s)
{
    const int d = a.d, B = w.batches;
    const int64_t P = a.run.paths;
    if (P > INT32_MAX) return cudaErrorInvalidValue;
    if (a.exact4) corr_wsum_kernel<true><<<grid, 128, 0, s>>>(a, w.Wbuf);
    else corr_wsum_kernel<false><<<grid, 128, 0, s>>>(a, w.Wbuf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Y = W Lhat^T: Y[p][a] = sum_b W[p][b] Lhat[a][b]
    if ((e = gemm_f32_abt(static_cast<int>(P), d, d, w.Wbuf, d, w.Ls, d, w.Ybuf, d, s)) != cudaSuccess) return e;
    const int64_t warps = (P < int64_t(1) << 20) ? P : (int64_t(1) << 20);
    corr_u_kernel<<<static_cast<int>((warps * 32 + 255) / 256), 256, 0, s>>>(a, w.drift, w.ws0, w.Ybuf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // H_b [d x d] = sum over batch b of u_p W_p^T
    if ((e = gemm_f32_atb_slices(d, d, static_cast<int>(P), w.Ybuf, d, w.Wbuf, d, w.kchunk, w.part, s)) != cudaSuccess)
        return e;
    const int64_t dd = static_cast<int64_t>(d) * d;
    const unsigned ge = static_cast<unsigned>(std::min<int64_t>((dd + 255) / 256, 1024));
    corr_lbar_kernel<<<dim3(ge, B + 1), 256, 0, s>>>(d, B, w.part, w.nb, w.cfac, w.out_dl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    corr_adj_a_kernel<<<dim3(ge, B + 1), 256, 0, s>>>(d, w.L, w.out_dl, w.Pm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned gr = static_cast<unsigned>((d + 7) / 8);  // 8 rows (columns) per block of 256
    corr_adj_x_kernel<<<dim3(gr, B + 1), 256, 0, s>>>(d, w.L, w.Pm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    corr_lt_kernel<<<ge, 256, 0, s>>>(d, w.L, w.Lt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    corr_adj_s_kernel<<<dim3(static_cast<unsigned>((d + 127) / 128), B + 1), 128, 0, s>>>(d, w.Lt, w.Pm, w.Sm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    corr_sym_kernel<<<dim3(ge, B + 1), 256, 0, s>>>(d, w.Sm, w.out_drho);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t dd2 = 2 * dd;
    corr_finish_kernel<<<static_cast<unsigned>((dd2 + 255) / 256), 256, 0, s>>>(d, B, w.nb, w.out_dl, w.out_drho,
                                                                              w.res_dl, w.res_drho);
    return cudaGetLastError();
}

}  // namespace gbmc
