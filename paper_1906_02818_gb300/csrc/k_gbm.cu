// Path-per-thread kernels for geometric Brownian motion (Eq. 1 with
// mu(X) = r X, sigma(X) = sigma X): the single-asset kernel (the scalar
// Euler-Maruyama scheme of Sec. II.A.1) and the dispatch of the FP32 basket
// kernels of k_basket.cuh.  The kernels fuse Philox4x32-10 + Box-Muller in
// registers, the state update, the payoff statistics and the reduction;
// nothing per path or per step touches global memory unless paths are
// materialised (mc_simulate).
#include "k_basket.cuh"

namespace gbmc {

namespace {

constexpr int kBlock = 256;

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

// Four uniforms of Philox block q of stream n (the same map as the normals).
__device__ __forceinline__ float4 uniforms4(uint64_t q, uint64_t n, const RoundKeys &rk)
{
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                             static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32)),
                                  rk);
    return make_float4(u01(x.x), u01(x.y), u01(x.z), u01(x.w));
}

constexpr uint64_t kBridgeDomain = uint64_t(1) << 56;  // stream of path n's bridge uniforms: 2^56 + n

// ------------------------------- 1-D GBM ---------------------------------
// BRIDGE (log-Euler only): continuous barrier monitoring.  Between grid values
// yp, y of log2(S/S0) the maximum of the Brownian bridge is drawn as
// (yp + y + sqrt((y - yp)^2 - cb lg2 U)) / 2 with cb = 2 dt sigma^2 log2(e)
// (Sec. VI.A.1; the formula in log2 units) and the minimum with the root
// subtracted; U = uniforms 2i and 2i + 1 of the bridge stream.  Eight
// blocks per SM (32 registers, an 8-byte spill): left free, the compiler
// takes 48 registers, 5 blocks fit, and the 2^20 x 64 call runs 76.3 us
// instead of 73.8 us.
template <int SCHEME, bool STATS, bool SAVE, bool BRIDGE>
__global__ void __launch_bounds__(kBlock, 8) gbm1d_kernel(const __grid_constant__ Gbm1dArgs a)
{
    __shared__ AccSlot s_acc[(kBlock / 32) * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];
    for (int i = threadIdx.x; i < (kBlock / 32) * a.pay.n * 2; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();

    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = a.run.steps;
    const float inv_m = 1.0f / static_cast<float>(M);
    for (int it = 0; it < a.run.ppt; ++it) {
        const int64_t nl = tid + it * gthreads;
        const bool valid = nl < a.run.paths;
        float uT = a.s0, avg = 0.0f;
        Stats st;
        st.init();
        if (valid) {
            const uint64_t n = static_cast<uint64_t>(a.run.path_offset + nl);
            float y = (SCHEME == MC_LOG_EULER) ? 0.0f : a.s0;  // log2(S/S0) or S
            float bmax = 0.0f, bmin = 0.0f;                    // bridge extremes of y
            const int64_t save_len = (static_cast<int64_t>(M / a.run.save_every) + 1) * a.run.paths;
            if (SAVE && GBMC_IN_BOUNDS(nl, save_len, kDbgGbm1dSave)) a.run.save[nl] = a.s0;
            const int nq = (M + 3) >> 2;
            for (int q = 0; q < nq; ++q) {
                const float4 z4 = normals4(static_cast<uint64_t>(q), n, a.run.rk);
                const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
                float4 ub[2];
                if (BRIDGE) {  // uniforms 8q .. 8q + 7: (max, min) of steps 4q .. 4q + 3
                    ub[0] = uniforms4(2 * static_cast<uint64_t>(q), kBridgeDomain + n, a.run.rk);
                    ub[1] = uniforms4(2 * static_cast<uint64_t>(q) + 1, kBridgeDomain + n, a.run.rk);
                }
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const int i = 4 * q + l;
                    if (i < M) {
                        const float yp = y;
                        if (SCHEME == MC_LOG_EULER) y += fmaf(a.b, zz[l], a.a);
                        else y = fmaf(y, fmaf(a.b, zz[l], a.a), y);
                        if (BRIDGE) {
                            const float4 u = ub[l >> 1];
                            const float umx = (l & 1) ? u.z : u.x, umn = (l & 1) ? u.w : u.y;
                            const float dy = y - yp, d2 = dy * dy;
                            const float rmax = sqrt_approx(fmaf(-a.cb, lg2_approx(umx), d2));
                            const float rmin = sqrt_approx(fmaf(-a.cb, lg2_approx(umn), d2));
                            bmax = fmaxf(bmax, 0.5f * (yp + y + rmax));
                            bmin = fminf(bmin, 0.5f * (yp + y - rmin));
                        }
                        if (STATS || SAVE) {
                            const float S = (SCHEME == MC_LOG_EULER) ? a.s0 * ex2_approx(y) : y;
                            if (STATS) st.add(S);
                            if (SAVE && ((i + 1) % a.run.save_every) == 0) {
                                const int64_t o = static_cast<int64_t>((i + 1) / a.run.save_every) * a.run.paths + nl;
                                if (GBMC_IN_BOUNDS(o, save_len, kDbgGbm1dSave)) a.run.save[o] = S;
                            }
                        }
                    }
                }
            }
            uT = (SCHEME == MC_LOG_EULER) ? a.s0 * ex2_approx(y) : y;
            avg = st.sum * inv_m;
            if (BRIDGE) {
                st.umax = a.s0 * ex2_approx(bmax);
                st.umin = a.s0 * ex2_approx(bmin);
            }
        }
        if (a.pay.n > 0) accumulate_payoffs(s_acc, a.pay, valid, uT, avg, st);
    }
    if (a.pay.n > 0) block_finish(s_acc, s_red, a.pay.n, a.red);
}

template <int SCHEME, bool STATS, bool SAVE, bool BRIDGE = false>
const void *gbm1d_fn()
{
    return reinterpret_cast<const void *>(&gbm1d_kernel<SCHEME, STATS, SAVE, BRIDGE>);
}

const void *gbm1d_select(const Gbm1dArgs &a)
{
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    const bool save = a.run.save != nullptr;
    if (a.scheme == MC_LOG_EULER) {
        if (save) return gbm1d_fn<MC_LOG_EULER, false, true>();
        if (a.bridge) return gbm1d_fn<MC_LOG_EULER, true, false, true>();
        return stats ? gbm1d_fn<MC_LOG_EULER, true, false>() : gbm1d_fn<MC_LOG_EULER, false, false>();
    }
    if (save) return gbm1d_fn<MC_EULER, false, true>();
    return stats ? gbm1d_fn<MC_EULER, true, false>() : gbm1d_fn<MC_EULER, false, false>();
}

template <int D>
const void *basket_select_d(const BasketArgs &a)
{
    return a.scheme == MC_LOG_EULER ? basket_select_scheme<D, MC_LOG_EULER>(a)
                                    : basket_select_scheme<D, MC_EULER>(a);
}

const void *basket_select(int D, const BasketArgs &a)
{
    switch (D) {
    case 4: return basket_select_d<4>(a);
    case 8: return basket_select_d<8>(a);
    case 16: return basket_select_d<16>(a);
    case 32: return basket_select_d<32>(a);
    case 64: return basket_select_d<64>(a);
    default: return nullptr;
    }
}

int occupancy_of(const void *fn, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

cudaError_t launch_gbm1d(const Gbm1dArgs &a, int grid, int block, cudaStream_t s)
{
    void *args[] = {const_cast<Gbm1dArgs *>(&a)};
    return cudaLaunchKernel(gbm1d_select(a), dim3(grid), dim3(block), args, 0, s);
}

int gbm1d_occupancy(const Gbm1dArgs &a, int block) { return occupancy_of(gbm1d_select(a), block); }

int basket_fp32_width(int d)
{
    for (int D : {4, 8, 16, 32, 64})
        if (d <= D) return D;
    return 0;
}

size_t basket_const_bytes(int D)
{
    switch (D) {
    case 4: return sizeof(BasketConst<4>);
    case 8: return sizeof(BasketConst<8>);
    case 16: return sizeof(BasketConst<16>);
    case 32: return sizeof(BasketConst<32>);
    case 64: return sizeof(BasketConst<64>);
    default: return 0;
    }
}

template <int D>
static void offsets_of(size_t *L, size_t *drift, size_t *ws0, size_t *w, size_t *s0)
{
    *L = offsetof(BasketConst<D>, Lp);
    *drift = offsetof(BasketConst<D>, drift);
    *ws0 = offsetof(BasketConst<D>, ws0);
    *w = offsetof(BasketConst<D>, w);
    *s0 = offsetof(BasketConst<D>, s0);
}

void basket_const_offsets(int D, size_t *L, size_t *drift, size_t *ws0, size_t *w, size_t *s0)
{
    switch (D) {
    case 4: offsets_of<4>(L, drift, ws0, w, s0); break;
    case 8: offsets_of<8>(L, drift, ws0, w, s0); break;
    case 16: offsets_of<16>(L, drift, ws0, w, s0); break;
    case 32: offsets_of<32>(L, drift, ws0, w, s0); break;
    default: offsets_of<64>(L, drift, ws0, w, s0); break;
    }
}

cudaError_t launch_basket_fp32(int D, const BasketArgs &a, const void *cst, int grid, int block,
                               cudaStream_t s)
{
    const void *fn = basket_select(D, a);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {const_cast<BasketArgs *>(&a), const_cast<void *>(cst)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, s);
}

int basket_fp32_occupancy(int D, const BasketArgs &a, int block)
{
    const void *fn = basket_select(D, a);
    return fn ? occupancy_of(fn, block) : 0;
}

}  // namespace gbmc
