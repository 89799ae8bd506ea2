// Pathwise (infinitesimal perturbation) Greeks (Sec. I.A.3; the paper's
// "Basket European option Delta" by back-propagation, Sec. VI.A.2).
//
//  * heston_adjoint_kernel — reverse mode.  The forward pass stores the path
//    state (log S / S0, v) every K steps in a checkpoint buffer
//    [segment][variable][thread] (coalesced across threads); the reverse
//    pass walks the segments backwards, recomputes each segment's states from
//    its checkpoint (the counter-based generator re-creates the same normals),
//    and back-propagates two adjoint vectors through the full-truncation
//    Euler step: one seeded by S_T (European kinds) and one by the
//    arithmetic average A (Asian kinds, injected at every monitoring date).
//    Because the sweep is linear in its seed, every European strike shares
//    the first and every Asian strike the second.
//  * gbm1d_greeks_kernel — single-asset GBM, log-Euler: the adjoint of
//    log S is constant along the path, so the sweep collapses to closed
//    forms in the forward pass (dS/dsigma = S (-sigma t + sqrt(dt) W_t)).
// Per path and payoff the kernels accumulate [price, Greek_1..Greek_G]
// (undiscounted; rho carries the -T f term) with the same warp / block /
// FP64 reduction as the pricers.
#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kBlock = 128;
constexpr int kMaxSeg = 64;  // checkpoint stride K <= 64 (states of a segment in local memory)

__device__ __forceinline__ float slope_of(int kind, float K, float uT, float avg)
{
    switch (kind) {
    case MC_CALL: return uT > K ? 1.0f : 0.0f;
    case MC_PUT: return K > uT ? -1.0f : 0.0f;
    case MC_ASIAN_CALL: return avg > K ? 1.0f : 0.0f;
    case MC_ASIAN_PUT: return K > avg ? -1.0f : 0.0f;
    default: return 0.0f;
    }
}

__device__ __forceinline__ bool is_asian(int kind) { return kind == MC_ASIAN_CALL || kind == MC_ASIAN_PUT; }

template <int NG>
__device__ __forceinline__ void accumulate_greeks(AccSlot *s_acc, const PayoffSet &pay, bool valid, float uT,
                                                  float avg, const float (&dE)[NG], const float (&dA)[NG],
                                                  int rho_slot, float T)
{
    const int nv = pay.n * (NG + 1);
    for (int p = 0; p < pay.n; ++p) {
        const float f = payoff_eval(pay.kind[p], pay.strike[p], INFINITY, uT, avg, 0.0f, 0.0f);
        const float g = slope_of(pay.kind[p], pay.strike[p], uT, avg);
        const bool as = is_asian(pay.kind[p]);
        warp_accumulate(s_acc, nv, p * (NG + 1), valid ? f : 0.0f);
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            float gk = g * (as ? dA[k] : dE[k]);
            if (k == rho_slot) gk -= T * f;
            warp_accumulate(s_acc, nv, p * (NG + 1) + 1 + k, valid ? gk : 0.0f);
        }
    }
}

// ------------------------------ 1-D GBM ----------------------------------
__global__ void __launch_bounds__(kBlock) gbm1d_greeks_kernel(const __grid_constant__ GreeksArgs a)
{
    extern __shared__ AccSlot s_acc[];
    __shared__ double s_red[32];
    const int nv = a.pay.n * 4;
    for (int i = threadIdx.x; i < (kBlock / 32) * nv * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();
    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = a.run.steps;
    const float inv_m = 1.0f / M;
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gthreads;
        const bool valid = nl < a.run.paths;
        float uT = 0.0f, avg = 0.0f;
        float dE[3] = {0.0f, 0.0f, 0.0f}, dA[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            float y = 0.0f, W = 0.0f, sS = 0.0f, sSt = 0.0f, sSW = 0.0f;
            for (int q = 0; q < (M + 3) / 4; ++q) {
                const float4 z4 = normals4(static_cast<uint64_t>(q), n, a.run.rk);
                const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const int i = 4 * q + l;
                    if (i < M) {
                        y += fmaf(a.b2, zz[l], a.a2);
                        W += zz[l];
                        const float S = a.s0w * ex2_approx(y);
                        const float t = (i + 1) * a.dt;
                        sS += S;
                        sSt = fmaf(S, t, sSt);
                        sSW = fmaf(S, W, sSW);
                    }
                }
            }
            uT = a.s0w * ex2_approx(y);
            avg = sS * inv_m;
            // European: d S_T / d(S0, sigma, r)
            dE[0] = uT / a.s0;
            dE[1] = uT * fmaf(-a.sigma, a.T, a.sdt * W);
            dE[2] = uT * a.T;
            // Asian: d A / d(S0, sigma, r)
            dA[0] = avg / a.s0;
            dA[1] = fmaf(-a.sigma, sSt, a.sdt * sSW) * inv_m;
            dA[2] = sSt * inv_m;
        }
        accumulate_greeks<3>(s_acc, a.pay, valid, uT, avg, dE, dA, 2, a.T);
    }
    block_finish(s_acc, s_red, nv, a.red);
}

// --------------------------- Heston adjoint --------------------------------
// Greek order: 0 S0, 1 v0, 2 r, 3 kappa, 4 theta, 5 xi, 6 rho.
__global__ void __launch_bounds__(kBlock) heston_adjoint_kernel(const __grid_constant__ GreeksArgs a)
{
    extern __shared__ AccSlot s_acc[];
    __shared__ double s_red[32];
    const int nv = a.pay.n * 8;
    for (int i = threadIdx.x; i < (kBlock / 32) * nv * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();
    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = a.run.steps, K = a.K;
    const int nseg = (M + K - 1) / K;
    const float dt = a.dt, inv_m = 1.0f / M;
    const float rho = a.rho, rhoc = a.rhoc, kap = a.kappa, th = a.theta, xi = a.xi;
    float xs[kMaxSeg], vs[kMaxSeg];
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gthreads;
        const bool valid = nl < a.run.paths;
        float uT = 0.0f, avg = 0.0f;
        float dE[7], dA[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) dE[k] = dA[k] = 0.0f;
        if (valid) {
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            NormalReader rd;
            rd.init(n, a.run.rk);
            // forward pass with checkpoints every K steps
            float x = 0.0f, v = a.v0, sS = 0.0f;
            for (int s = 0; s < nseg; ++s) {
                if (GBMC_IN_BOUNDS((static_cast<int64_t>(s) * 2 + 1) * gthreads + tid,
                                   static_cast<int64_t>(nseg) * 2 * gthreads, kDbgCkptStore)) {
                    a.ckpt[(static_cast<int64_t>(s) * 2) * gthreads + tid] = x;
                    a.ckpt[(static_cast<int64_t>(s) * 2 + 1) * gthreads + tid] = v;
                }
                const int e = min(M, (s + 1) * K);
                for (int i = s * K; i < e; ++i) {
                    const float z1 = rd.get(2 * static_cast<uint64_t>(i));
                    const float z2 = rd.get(2 * static_cast<uint64_t>(i) + 1);
                    const float vp = fmaxf(v, 0.0f);
                    const float sq = sqrt_approx(vp * dt);
                    const float c = fmaf(rho, z1, rhoc * z2);
                    x += fmaf(sq, c, (a.r - 0.5f * vp) * dt);
                    v += fmaf(xi * sq, z1, kap * (th - vp) * dt);
                    sS += a.s0w * ex2_approx(x * kLog2e);
                }
            }
            uT = a.s0w * ex2_approx(x * kLog2e);
            avg = sS * inv_m;
            // reverse pass: adjoints of (x, v) for the seeds S_T and A
            const float lx = uT;  // d S_T / d x_i is S_T at every i
            float lv = 0.0f, mx = uT * inv_m, mv = 0.0f;
            float gEr = 0, gEk = 0, gEt = 0, gEx = 0, gEp = 0, gAr = 0, gAk = 0, gAt = 0, gAx = 0, gAp = 0;
            for (int s = nseg - 1; s >= 0; --s) {
                float xc = 0.0f, vc = 0.0f;
                if (GBMC_IN_BOUNDS((static_cast<int64_t>(s) * 2 + 1) * gthreads + tid,
                                   static_cast<int64_t>(nseg) * 2 * gthreads, kDbgCkptLoad)) {
                    xc = a.ckpt[(static_cast<int64_t>(s) * 2) * gthreads + tid];
                    vc = a.ckpt[(static_cast<int64_t>(s) * 2 + 1) * gthreads + tid];
                }
                const int b = s * K, e = min(M, (s + 1) * K);
                for (int i = b; i < e; ++i) {  // recompute the segment's states
                    xs[i - b] = xc;
                    vs[i - b] = vc;
                    const float z1 = rd.get(2 * static_cast<uint64_t>(i));
                    const float z2 = rd.get(2 * static_cast<uint64_t>(i) + 1);
                    const float vp = fmaxf(vc, 0.0f);
                    const float sq = sqrt_approx(vp * dt);
                    const float c = fmaf(rho, z1, rhoc * z2);
                    xc += fmaf(sq, c, (a.r - 0.5f * vp) * dt);
                    vc += fmaf(xi * sq, z1, kap * (th - vp) * dt);
                }
                for (int i = e - 1; i >= b; --i) {  // back-propagate through step i
                    const float z1 = rd.get(2 * static_cast<uint64_t>(i));
                    const float z2 = rd.get(2 * static_cast<uint64_t>(i) + 1);
                    const float vi = vs[i - b];
                    const float vp = fmaxf(vi, 0.0f);
                    const float sq = sqrt_approx(vp * dt);
                    const float c = fmaf(rho, z1, rhoc * z2);
                    const float dsq = vp > 0.0f ? 0.5f * dt / sq : 0.0f;
                    const float dcr = z1 - rho / rhoc * z2;
                    gEr = fmaf(lx, dt, gEr);
                    gEk = fmaf(lv, (th - vp) * dt, gEk);
                    gEt = fmaf(lv, kap * dt, gEt);
                    gEx = fmaf(lv, sq * z1, gEx);
                    gEp = fmaf(lx, sq * dcr, gEp);
                    gAr = fmaf(mx, dt, gAr);
                    gAk = fmaf(mv, (th - vp) * dt, gAk);
                    gAt = fmaf(mv, kap * dt, gAt);
                    gAx = fmaf(mv, sq * z1, gAx);
                    gAp = fmaf(mx, sq * dcr, gAp);
                    if (vi > 0.0f) {
                        const float ax = fmaf(c, dsq, -0.5f * dt);
                        const float av = fmaf(xi * z1, dsq, -kap * dt);
                        lv = fmaf(lx, ax, fmaf(lv, av, lv));
                        mv = fmaf(mx, ax, fmaf(mv, av, mv));
                    }
                    if (i >= 1) mx = fmaf(a.s0w * ex2_approx(xs[i - b] * kLog2e), inv_m, mx);
                }
            }
            dE[0] = uT / a.s0; dE[1] = lv; dE[2] = gEr; dE[3] = gEk; dE[4] = gEt; dE[5] = gEx; dE[6] = gEp;
            dA[0] = avg / a.s0; dA[1] = mv; dA[2] = gAr; dA[3] = gAk; dA[4] = gAt; dA[5] = gAx; dA[6] = gAp;
        }
        accumulate_greeks<7>(s_acc, a.pay, valid, uT, avg, dE, dA, 2, a.T);
    }
    block_finish(s_acc, s_red, nv, a.red);
}

}  // namespace

const void *greeks_kernel(int model) {
    return model == MC_HESTON ? reinterpret_cast<const void *>(&heston_adjoint_kernel)
                              : reinterpret_cast<const void *>(&gbm1d_greeks_kernel);
}

size_t greeks_smem(int model, int n_payoff)
{
    const int per = model == MC_HESTON ? 8 : 4;
    return static_cast<size_t>(kBlock / 32) * n_payoff * per * 2 * sizeof(AccSlot);
}

int greeks_block() { return kBlock; }

cudaError_t launch_greeks(const GreeksArgs &a, int grid, cudaStream_t s)
{
    const void *fn = greeks_kernel(a.model);
    const size_t smem = greeks_smem(a.model, a.pay.n);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<GreeksArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, smem, s);
}

int greeks_occupancy(int model, int n_payoff)
{
    const void *fn = greeks_kernel(model);
    const size_t smem = greeks_smem(model, n_payoff);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBlock, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace gbmc
