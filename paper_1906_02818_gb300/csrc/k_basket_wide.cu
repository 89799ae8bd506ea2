// FP32 contraction for large baskets (64 < d <= 512), the reference
// precision of the tensor-core kernels: the multivariate Euler step of
// Sec. II.A.2 for a tile of 64 paths as a register-tiled SIMT product.
//   * CTA = 64 paths x D assets (D = 128, 256 or 512, zero-padded), 512
//     threads; thread (pg, ag) owns paths 4 pg .. 4 pg + 3 and the assets
//     128 j + 4 ag .. + 3 (j < D / 128): 4 x D / 32 running sums in registers
//     as asset pairs, acc[p][a] = sum over steps of (Lhat z)_a, Lhat =
//     log2(e) sqrt(dt) diag(sigma) Lrho, accumulated by packed FP32x2 FMAs
//     (one instruction for two assets of one path; each lane an FP32 fma).
//   * per step: the CTA draws the 64 x d normals into shared memory
//     (z[k][path], consecutive threads on consecutive paths), then streams
//     Lhat^T in chunks of 16 rows (cp.async double buffer) and accumulates;
//     128-asset blocks that lie above the chunk (zero in the lower-triangular
//     factor) are skipped.
//   * at the end of the tile: log2(S_a / S0_a) = M drift_a + acc, the basket,
//     European payoffs and the pathwise delta / vega / rho of payoff 0.
#include "mc_kernels.cuh"

namespace gbmc {
namespace {

constexpr int kP = 64;       // paths per CTA
constexpr int kThreads = 512;
constexpr int kKC = 16;      // factor rows per chunk

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Element e (0..3) of a thread's four consecutive assets held as two pairs.
__device__ __forceinline__ float accel(const f32x2 *pr, int e) { return (e & 1) ? hi_of(pr[e >> 1]) : lo_of(pr[e >> 1]); }

template <int D>
__global__ void __launch_bounds__(kThreads, 1) basket_wide_kernel(const __grid_constant__ BigArgs a)
{
    constexpr int J = D / 128;  // 4-asset groups per thread
    extern __shared__ __align__(16) float sm[];
    float *zs = sm;                      // [D][kP]
    float *Ls = sm + D * kP;             // [2][kKC][D]
    __shared__ float s_pay[MC_MAX_PAYOFFS][2];
    __shared__ float s_g[kBigMaxD * 2 + 1][2];
    __shared__ float s_u[kP];
    const int t = threadIdx.x, lane = t & 31;
    const int pg = t >> 5, ag = t & 31;  // a warp = one path group, 32 asset groups
    const int d = a.d, nv = a.pay.n, M = a.run.steps;
    for (int i = t; i < nv * 2; i += kThreads) s_pay[i >> 1][i & 1] = 0.0f;
    for (int i = t; i < (2 * d + 1) * 2; i += kThreads) s_g[i >> 1][i & 1] = 0.0f;
    const int64_t ntiles = (a.run.paths + kP - 1) / kP;
    const int nchunks = (d + kKC - 1) / kKC;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        f32x2 acc2[4][J][2];  // [path][asset group][asset pair]
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int j = 0; j < J; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) acc2[p][j][e] = pack2(0.0f, 0.0f);
        // RNG mapping: path t % 64, normals [q*D/8, (q+1)*D/8) with q = t / 64
        const int rp = t & (kP - 1), rq = t >> 6;
        const int64_t rnl = tile * kP + rp;
        const bool rvalid = rnl < a.run.paths;
        const uint64_t rn = static_cast<uint64_t>(a.run.path_offset + (rvalid ? rnl : 0));
        NormalReader rd;
        rd.init(rn, a.run.rk);
        for (int i = 0; i < M; ++i) {
            __syncthreads();  // previous step done with zs
            for (int k = rq * (D / 8); k < (rq + 1) * (D / 8); k += 4) {
                float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                if (rvalid && k < d) {
                    if (a.exact4) {
                        z = normals4((static_cast<uint64_t>(i) * d + k) >> 2, rn, a.run.rk);
                    } else {
                        const uint64_t j0 = static_cast<uint64_t>(i) * d + k;
                        z.x = rd.get(j0);
                        z.y = k + 1 < d ? rd.get(j0 + 1) : 0.f;
                        z.z = k + 2 < d ? rd.get(j0 + 2) : 0.f;
                        z.w = k + 3 < d ? rd.get(j0 + 3) : 0.f;
                    }
                }
                zs[(k + 0) * kP + rp] = z.x;
                zs[(k + 1) * kP + rp] = z.y;
                zs[(k + 2) * kP + rp] = z.z;
                zs[(k + 3) * kP + rp] = z.w;
            }
            // first factor chunk
            for (int e = t * 4; e < kKC * D; e += kThreads * 4) cp_async16(Ls + e, a.Lp + e);
            cp_async_commit();
            for (int c = 0; c < nchunks; ++c) {
                cp_async_wait_all();
                __syncthreads();  // chunk c (and, at c = 0, the normals) visible
                const float *Lc = Ls + (c & 1) * kKC * D;
                if (c + 1 < nchunks) {  // prefetch the next chunk into the other buffer
                    float *dst = Ls + ((c + 1) & 1) * kKC * D;
                    const float *src = a.Lp + static_cast<size_t>(c + 1) * kKC * D;
                    for (int e = t * 4; e < kKC * D; e += kThreads * 4) cp_async16(dst + e, src + e);
                    cp_async_commit();
                }
                const int k0 = c * kKC;
#pragma unroll 4
                for (int kk = 0; kk < kKC; ++kk) {
                    const float4 zv = *reinterpret_cast<const float4 *>(zs + (k0 + kk) * kP + 4 * pg);
                    const f32x2 zz[4] = {pack2(zv.x, zv.x), pack2(zv.y, zv.y), pack2(zv.z, zv.z), pack2(zv.w, zv.w)};
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        if (128 * j + 127 < k0) continue;  // block above the diagonal chunk: zero
                        const ulonglong2 lv = *reinterpret_cast<const ulonglong2 *>(Lc + kk * D + 128 * j + 4 * ag);
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            acc2[p][j][0] = ffma2(lv.x, zz[p], acc2[p][j][0]);
                            acc2[p][j][1] = ffma2(lv.y, zz[p], acc2[p][j][1]);
                        }
                    }
                }
                __syncthreads();  // everyone done with chunk c before it is overwritten
            }
        }
        // ---- epilogue ----
        float Ux[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = 128 * j + 4 * ag + e;
                if (col < d) {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        Ux[p] = fmaf(a.ws0[col], ex2_approx(fmaf(static_cast<float>(M), a.drift[col], accel(acc2[p][j], e))), Ux[p]);
                }
            }
        // sum over the 32 asset groups of each path (the lanes of one warp)
#pragma unroll
        for (int p = 0; p < 4; ++p) Ux[p] = warp_sum(Ux[p]);
        if (ag == 0)
#pragma unroll
            for (int p = 0; p < 4; ++p) s_u[4 * pg + p] = Ux[p];
        __syncthreads();
        if (t < kP) {  // payoffs, one thread per path
            const bool valid = tile * kP + t < a.run.paths;
            for (int q = 0; q < nv; ++q) {
                const float f = valid ? payoff_eval(a.pay.kind[q], a.pay.strike[q], INFINITY, s_u[t], 0.f, 0.f, 0.f) : 0.f;
                const float s1 = warp_sum(f), s2 = warp_sum(f * f);
                if (lane == 0) {
                    atomicAdd(&s_pay[q][0], s1);
                    atomicAdd(&s_pay[q][1], s2);
                }
            }
        }
        if (a.greeks) {
            float gs[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float U = s_u[4 * pg + p];
                const bool valid = tile * kP + 4 * pg + p < a.run.paths;
                gs[p] = valid ? (a.pay.kind[0] == MC_PUT ? (U < a.pay.strike[0] ? -1.f : 0.f)
                                                         : (U > a.pay.strike[0] ? 1.f : 0.f))
                              : 0.f;
            }
#pragma unroll
            for (int j = 0; j < J; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int col = 128 * j + 4 * ag + e;
                    float d1 = 0.f, d2 = 0.f, v1 = 0.f, v2 = 0.f;
                    if (col < d) {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float S = a.s0[col] * ex2_approx(fmaf(static_cast<float>(M), a.drift[col], accel(acc2[p][j], e)));
                            const float dl = gs[p] * a.w[col] * S / a.s0[col];
                            // sqrt(dt) (Lrho W)_col = acc / (log2(e) sigma_col)
                            const float vg = gs[p] * a.w[col] * S * fmaf(-a.sigma[col], a.T, accel(acc2[p][j], e) / (kLog2e * a.sigma[col]));
                            d1 += dl; d2 += dl * dl; v1 += vg; v2 += vg * vg;
                        }
                    }
                    // each lane holds its own columns: one atomic per (warp, column)
                    if (col < d) {
                        atomicAdd(&s_g[col][0], d1);
                        atomicAdd(&s_g[col][1], d2);
                        atomicAdd(&s_g[d + col][0], v1);
                        atomicAdd(&s_g[d + col][1], v2);
                    }
                }
            if (t < kP) {
                const float U = s_u[t];
                const bool valid = tile * kP + t < a.run.paths;
                const float g = valid ? (a.pay.kind[0] == MC_PUT ? (U < a.pay.strike[0] ? -1.f : 0.f)
                                                                 : (U > a.pay.strike[0] ? 1.f : 0.f))
                                      : 0.f;
                const float f = valid ? payoff_eval(a.pay.kind[0], a.pay.strike[0], INFINITY, U, 0.f, 0.f, 0.f) : 0.f;
                const float rr = g * U * a.T - a.T * f;
                const float r1 = warp_sum(rr), r2 = warp_sum(rr * rr);
                if (lane == 0) {
                    atomicAdd(&s_g[2 * d][0], r1);
                    atomicAdd(&s_g[2 * d][1], r2);
                }
            }
        }
        __syncthreads();
    }
    // per-CTA partials -> FP64 sum by the last CTA
    const int nvals = nv + (a.greeks ? 2 * d + 1 : 0);
    for (int i = t; i < nvals * 2; i += kThreads) {
        const int k = i >> 1, m = i & 1;
        a.partials[static_cast<size_t>(blockIdx.x) * nvals * 2 + i] = k < nv ? s_pay[k][m] : s_g[k - nv][m];
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int s_last;
    if (t == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double N = static_cast<double>(a.run.paths);
    for (int k = t; k < nvals; k += kThreads) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < static_cast<int>(gridDim.x); ++b) {
            s1 += a.partials[static_cast<size_t>(b) * nvals * 2 + 2 * k];
            s2 += a.partials[static_cast<size_t>(b) * nvals * 2 + 2 * k + 1];
        }
        const double mean = s1 / N, var = fmax(s2 / N - mean * mean, 0.0);
        mc_result r;
        r.price = a.disc * mean;
        r.se = a.run.paths > 1 ? a.disc * sqrt(var / (N - 1.0)) : 0.0;
        a.out[k] = r;
    }
    __syncthreads();
    if (t == 0) *a.ticket = 0u;
}

// LT[k][a] (D x D, k-major) = log2(e) sqrt(dt) sigma_a Lrho[a][k] (0 above the
// diagonal and beyond d); drift[a] = log2(e) (r - sigma_a^2 / 2) dt.
__global__ void wide_prep_kernel(int d, int D, const double *L, const double *sigma, double sdt, double r, double dt,
                                 float *LT, float *drift)
{
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < static_cast<int64_t>(D) * D;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(idx / D), col = static_cast<int>(idx % D);
        double v = 0.0;
        if (col < d && k <= col) v = M_LOG2E * sdt * sigma[col] * L[static_cast<int64_t>(col) * d + k];
        LT[idx] = static_cast<float>(v);
    }
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < d; col += gridDim.x * blockDim.x)
        drift[col] = static_cast<float>(M_LOG2E * (r - 0.5 * sigma[col] * sigma[col]) * dt);
}

}  // namespace

int wide_width(int d) { return d <= 128 ? 128 : (d <= 256 ? 256 : 512); }

size_t wide_smem(int D) { return static_cast<size_t>(D) * kP * sizeof(float) + 2 * kKC * static_cast<size_t>(D) * sizeof(float); }

const void *basket_wide_fn(int D)
{
    switch (D) {
    case 128: return reinterpret_cast<const void *>(&basket_wide_kernel<128>);
    case 256: return reinterpret_cast<const void *>(&basket_wide_kernel<256>);
    default: return reinterpret_cast<const void *>(&basket_wide_kernel<512>);
    }
}

int basket_wide_block() { return kThreads; }

cudaError_t launch_wide_prep(int d, const double *L, const double *sigma, double sdt, double r, double dt, float *LT,
                             float *drift, cudaStream_t s)
{
    const int D = wide_width(d);
    wide_prep_kernel<<<256, 256, 0, s>>>(d, D, L, sigma, sdt, r, dt, LT, drift);
    return cudaGetLastError();
}

}  // namespace gbmc
