// FP32 contraction for large baskets (64 < d <= 512), the reference
// precision of the tensor-core kernels: one thread per path, the state and
// the step's normals in thread-local memory (they do not fit registers), the
// packed factor c sqrt(dt) diag(sigma) Lrho read from global memory (every
// thread of a warp reads the same entry: one broadcast load), the
// multivariate Euler step of Sec. II.A.2 row by row.  European payoffs on
// U(T) and the pathwise Greeks of payoff 0, accumulated per CTA with shared
// atomics and finished in FP64 by the last CTA.
#include "mc_kernels.cuh"

namespace gbmc {
namespace {

constexpr int kBlock = 128;

__global__ void __launch_bounds__(kBlock) basket_wide_kernel(const BigArgs a)
{
    __shared__ float s_pay[MC_MAX_PAYOFFS][2];
    __shared__ float s_g[kBigMaxD * 2 + 1][2];
    const int d = a.d, nv = a.pay.n;
    for (int i = threadIdx.x; i < nv * 2; i += blockDim.x) s_pay[i >> 1][i & 1] = 0.0f;
    for (int i = threadIdx.x; i < (2 * d + 1) * 2; i += blockDim.x) s_g[i >> 1][i & 1] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t ppt = (a.run.paths + gthreads - 1) / gthreads;
    const int M = a.run.steps;
    float x[kBigMaxD], z[kBigMaxD];
    for (int64_t it = 0; it < ppt; ++it) {
        const int64_t nl = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x + it * gthreads;
        const bool valid = nl < a.run.paths;
        float U = 0.0f;
        if (valid) {
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            NormalReader rd;
            rd.init(n, a.run.k0, a.run.k1);
            for (int j = 0; j < d; ++j) x[j] = 0.0f;
            for (int i = 0; i < M; ++i) {
                for (int j = 0; j < d; ++j) z[j] = rd.get(static_cast<uint64_t>(i) * d + j);
                for (int j = 0; j < d; ++j) {
                    const float *row = a.Lp + static_cast<int64_t>(j) * (j + 1) / 2;
                    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
                    int k = 0;
                    for (; k + 3 <= j; k += 4) {
                        s0 = fmaf(row[k], z[k], s0);
                        s1 = fmaf(row[k + 1], z[k + 1], s1);
                        s2 = fmaf(row[k + 2], z[k + 2], s2);
                        s3 = fmaf(row[k + 3], z[k + 3], s3);
                    }
                    for (; k <= j; ++k) s0 = fmaf(row[k], z[k], s0);
                    x[j] += a.drift[j] + ((s0 + s1) + (s2 + s3));
                }
            }
            for (int j = 0; j < d; ++j) U = fmaf(a.ws0[j], ex2_approx(x[j]), U);
        }
        for (int p = 0; p < nv; ++p) {
            const float f = valid ? payoff_eval(a.pay.kind[p], a.pay.strike[p], INFINITY, U, 0.0f, 0.0f, 0.0f) : 0.0f;
            const float s1 = warp_sum(f), s2 = warp_sum(f * f);
            if (lane == 0) {
                atomicAdd(&s_pay[p][0], s1);
                atomicAdd(&s_pay[p][1], s2);
            }
        }
        if (a.greeks) {
            const float g = valid ? (a.pay.kind[0] == MC_PUT ? (U < a.pay.strike[0] ? -1.0f : 0.0f)
                                                             : (U > a.pay.strike[0] ? 1.0f : 0.0f))
                                  : 0.0f;
            for (int j = 0; j < d; ++j) {
                const float S = valid ? a.s0[j] * ex2_approx(x[j]) : 0.0f;
                // sqrt(dt) (Lrho W)_j = (x_j - M drift_j) / (log2(e) sigma_j)
                const float bw = valid ? (x[j] - M * a.drift[j]) / (kLog2e * a.sigma[j]) : 0.0f;
                const float dl = g * a.w[j] * S / a.s0[j];
                const float vg = g * a.w[j] * S * fmaf(-a.sigma[j], a.T, bw);
                const float d1 = warp_sum(dl), d2 = warp_sum(dl * dl), v1 = warp_sum(vg), v2 = warp_sum(vg * vg);
                if (lane == 0) {
                    atomicAdd(&s_g[j][0], d1);
                    atomicAdd(&s_g[j][1], d2);
                    atomicAdd(&s_g[d + j][0], v1);
                    atomicAdd(&s_g[d + j][1], v2);
                }
            }
            const float f = valid ? payoff_eval(a.pay.kind[0], a.pay.strike[0], INFINITY, U, 0.0f, 0.0f, 0.0f) : 0.0f;
            const float rr = g * U * a.T - a.T * f;
            const float r1 = warp_sum(rr), r2 = warp_sum(rr * rr);
            if (lane == 0) {
                atomicAdd(&s_g[2 * d][0], r1);
                atomicAdd(&s_g[2 * d][1], r2);
            }
        }
    }
    __syncthreads();
    const int nvals = nv + (a.greeks ? 2 * d + 1 : 0);
    for (int i = threadIdx.x; i < nvals * 2; i += blockDim.x) {
        const int k = i >> 1, m = i & 1;
        a.partials[static_cast<size_t>(blockIdx.x) * nvals * 2 + i] = k < nv ? s_pay[k][m] : s_g[k - nv][m];
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int s_last;
    if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double N = static_cast<double>(a.run.paths);
    for (int k = threadIdx.x; k < nvals; k += blockDim.x) {
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
    if (threadIdx.x == 0) *a.ticket = 0u;
}

}  // namespace

const void *basket_wide_fn() { return reinterpret_cast<const void *>(&basket_wide_kernel); }
int basket_wide_block() { return kBlock; }

}  // namespace gbmc
