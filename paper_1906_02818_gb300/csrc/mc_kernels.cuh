// Launch-parameter blocks and host launchers of the path kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mc_device.cuh"

#include <nvtx3/nvToolsExt.h>

#include "mc_debug.cuh"

namespace gbmc {

// A named NVTX range around a host phase of an entry point (set-up, launch,
// read-back), for timeline profilers; header-only, inert unless a profiler
// attaches.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Common per-launch fields of every path kernel.
struct PathRun {
    int64_t paths;        // paths of this launch
    int64_t path_offset;  // global index of the first one
    uint32_t k0, k1;      // Philox key
    RoundKeys rk;         // its ten round keys (set_seed)
    int steps;
    int ppt;              // paths per thread (grid-stride count)
    float *save;          // mc_simulate output or nullptr
    int save_every;
};

// Key (seed lo, seed hi) and its round keys.
inline void set_seed(PathRun &r, uint64_t seed)
{
    r.k0 = static_cast<uint32_t>(seed);
    r.k1 = static_cast<uint32_t>(seed >> 32);
    r.rk = round_keys(r.k0, r.k1);
}

// Single-asset GBM.  log-Euler: y = log2(S/S0) += a + b z with
// a = log2(e) (r - sigma^2/2) dt, b = log2(e) sigma sqrt(dt).
// Euler: S <- S + S (a + b z) with a = r dt, b = sigma sqrt(dt).
struct Gbm1dArgs {
    PathRun run;
    int scheme;
    float s0, a, b;
    int bridge;   // continuous monitoring via the Brownian-bridge extremes (log-Euler)
    float cb;     // 2 dt sigma^2 log2(e): squared bridge spread term per -lg2(U)
    PayoffSet pay;
    ReduceArgs red;
};

// Correlated basket of at most D assets (D even) with the Cholesky factor in
// the launch-parameter block (constant bank): the lower triangle of
// Lhat = c sqrt(dt) diag(sigma) Lrho (c = log2(e) for log-Euler, 1 for Euler)
// as column pairs for packed FP32x2 FMAs: column k holds the row pairs
// (2q, 2q + 1), q = k/2 .. D/2 - 1, low half row 2q, at pair
// basket_pair_base(D, k) + q - k/2 (row 2q = k - 1 of the first pair is the
// zero above the diagonal).  Entries for assets >= d are zero.
__host__ __device__ constexpr int basket_pair_count(int D) { return D * D / 4 + D / 2; }
__host__ __device__ constexpr int basket_pair_base(int D, int k)
{
    // sum over k' < k of (D/2 - floor(k'/2))
    return k * (D / 2) - (k / 2) * ((k / 2) - 1) - ((k & 1) ? k / 2 : 0);
}
template <int D>
struct BasketConst {
    unsigned long long Lp[basket_pair_count(D)];
    float drift[D];  // log-Euler: log2(e) (r - sigma_a^2/2) dt; Euler: r dt
    float ws0[D];    // w_a * S0_a
    float w[D];
    float s0[D];
};

struct BasketArgs {
    PathRun run;
    int d;
    int scheme;
    PayoffSet pay;
    ReduceArgs red;
};

// Heston full-truncation Euler, y = log2(S/S0).
struct HestonArgs {
    PathRun run;
    float s0, v0, r, kappa, theta, xi, rho, rhoc, dt;
    PayoffSet pay;
    ReduceArgs red;
};

// Tensor-core basket (d <= 64, padded to 64): launch-parameter constants per
// asset column n and the per-launch arguments.
struct TcConst {
    float drift[64];  // log-Euler: log2(e) (r - sigma_n^2/2) dt; Euler: r dt
    float cs[64];     // scale of column n of the MMA result: c sqrt(dt) sigma_n / s_n
    float ws0[64];    // w_n S0_n
    float w[64];
    float s0[64];
};

struct TcArgs {
    PathRun run;
    int d;
    int scheme;
    const uint8_t *bimg;   // pre-swizzled quantised factor tile (device)
    PayoffSet pay;
    ReduceArgs red;
    unsigned int *err;     // set to 1 when a bounded wait gave up
    uint32_t wait_cap;     // polls per mbarrier wait before giving up
    uint32_t stall;        // test request: fail through a wait nothing completes (GBMC_TEST_STALL)
};

// Large baskets (k_basket_big.cuh, tensor cores; k_basket_wide.cu, FP32):
// d <= kBigMaxD, European payoffs on U(T), optional pathwise Greeks of
// payoff 0 (delta_n, vega_n, rho).  Per-column arrays are device pointers.
constexpr int kBigMaxD = 512;
struct BigArgs {
    PathRun run;
    int d;
    int exact4;             // d % 4 == 0: each 16-normal group is 4 whole Philox blocks
    int greeks;
    const uint8_t *bimg;    // tensor cores: pre-swizzled factor chunks
    const float *Lp;        // FP32: k-major dense log2(e) sqrt(dt) diag(sigma) Lrho, [D x D]
    const float *cs, *mdrift, *vscale;  // tensor cores: epilogue constants per column
    const float *drift;     // FP32: per-step drift (log2 units)
    const float *ws0, *w, *s0, *sigma;
    float T, sdt;
    PayoffSet pay;
    float *partials;        // [grid][n_values][2]
    unsigned int *ticket;
    mc_result *out;         // [n_payoff (+ 2d + 1)]
    unsigned int *err;
    double disc;
    uint32_t wait_cap;
};
cudaError_t launch_basket_big(int prec, const BigArgs &a, int grid, cudaStream_t s);
int basket_big_grid(int prec, int64_t paths);
cudaError_t launch_big_prep(int prec, int d, const double *L, const double *sigma, double cfac, double sdt, double r,
                            double dt, int M, uint8_t *bimg, float *cs, float *mdrift, float *vscale, cudaStream_t s);
// FP32 large baskets: dense k-major factor LT [D x D], D = wide_width(d).
int wide_width(int d);
cudaError_t launch_wide_prep(int d, const double *L, const double *sigma, double sdt, double r, double dt, float *LT,
                             float *drift, cudaStream_t s);
size_t big_bimg_bytes(int prec);

// Pathwise Greeks (k_greeks.cu): single-asset GBM (log-Euler, closed forms)
// and Heston (reverse-mode adjoint with checkpoints every K steps).
struct GreeksArgs {
    PathRun run;
    int model;          // MC_GBM (d = 1) or MC_HESTON
    float s0;           // S0 (denominator of delta)
    float s0w;          // w * S0: the monitored underlying is U = w S
    float sigma, r, dt, sdt, T;
    float a2, b2;       // GBM: log2(S/S0) += a2 + b2 z
    float v0, kappa, theta, xi, rho, rhoc;
    int K;              // Heston checkpoint stride (1..64)
    float *ckpt;        // Heston: [ceil(M/K)][2][grid * block] checkpoint buffer
    PayoffSet pay;      // European / Asian kinds only
    ReduceArgs red;     // n_payoff * (1 + G) values per path
};
cudaError_t launch_greeks(const GreeksArgs &a, int grid, cudaStream_t s);
int greeks_occupancy(int model, int n_payoff);
int greeks_block();

// Correction level of the two-level precision estimator (k_mlmc.cu): d <= 64
// padded to 64; the FP32 factor Lhat and the dequantised tensor-core factor
// Lq (packed lower triangles), Lq's column scales, drift and weights.
constexpr int kMlmcMaxPayoffs = 10;  // 3 accumulated values per payoff
struct MlmcConst {
    // the FP32 factor and its tensor-core rounding as column pairs (the
    // BasketConst<64> layout: column k's pairs q >= k/2 at basket_pair_base),
    // 64-bit operands of the packed FMAs; zero above the diagonal and beyond d
    unsigned long long Lp[basket_pair_count(64)];
    unsigned long long Lqp[basket_pair_count(64)];
    float csq[64];
    float drift[64];
    float ws0[64];
    float w[64];
    float s0[64];
};
struct MlmcArgs {
    PathRun run;
    int d;
    int scheme;
    PayoffSet pay;
    ReduceArgs red;  // 3 n_payoff values: f_fp32 - f_q, f_fp32, f_q
};
cudaError_t launch_mlmc_prep(int prec, int d, const double *L, const double *sigma, double cfac, double sdt,
                             float *Lq, float *csq, cudaStream_t s);
cudaError_t launch_mlmc_coupled(int prec, const MlmcArgs &a, const MlmcConst &c, int grid, cudaStream_t s);
int mlmc_occupancy(int prec, const MlmcArgs &a);
int mlmc_block();
int mlmc_paths_per_block();  // paths a block carries at a time (the grid's unit)

// Randomised quasi-Monte Carlo (k_qmc.cu): Sobol direction words of up to
// kQmcMaxDims dimensions, the FP32 factor Lhat (packed, rows of width
// kQmcMaxAssets) and the basket constants; d <= 32 and 2 d M <= 64.
constexpr int kQmcMaxDims = 64;
constexpr int kQmcMaxAssets = 32;
struct QmcConst {
    uint32_t V[kQmcMaxDims][32];
    float L[kQmcMaxAssets * (kQmcMaxAssets + 1) / 2];
    float drift[kQmcMaxAssets];
    float ws0[kQmcMaxAssets];
    float w[kQmcMaxAssets];
    float s0[kQmcMaxAssets];
};
struct QmcArgs {
    int64_t n0, npts;   // first point index, points per replication
    int steps, d, scheme, ndim, reps;
    uint32_t k0, k1;    // Philox key of the digital shifts
    RoundKeys rk;       // its round keys
    PayoffSet pay;
    double *sums;       // [reps][n_payoff] undiscounted payoff totals (zero on entry)
};
void qmc_directions(int ndim, uint32_t (*V)[32]);
cudaError_t launch_qmc(const QmcArgs &a, const QmcConst &c, int grid, cudaStream_t s);
int qmc_occupancy(const QmcArgs &a);
int qmc_block();

// Factor-model GBM basket (k_factor.cu): device arrays padded to 256 G
// assets (G = ceil(d / 256) warps per 4 paths): B' [k][256 G] =
// c sqrt(dt) sigma_a B_aj, e' = c sqrt(dt) sigma_a e_a, drift, w S0, w, S0
// (padded assets: zero B', e', weights; S0 = 1).
constexpr int kFactorMax = 16;
constexpr int kFactorMaxD = 512;
struct FactorArgs {
    PathRun run;
    int d, k, G, scheme;
    int exact4;  // k % 4 == 0 and d % 4 == 0: aligned Philox blocks
    const float *Bp, *ep, *drift, *ws0, *w, *s0;
    PayoffSet pay;
    ReduceArgs red;
    // Pathwise Greeks (log-Euler, one European call or put): per-CTA sums of
    // the undiscounted per-path delta_a, vega_a (a < d) and rho terms and
    // of their squares, gpart [grid][2d + 1][2].
    int greeks;
    const float *sigma;  // [256 G]
    float T, r;
    float *gpart;
};
// Means and standard errors of the Greeks from gpart (FP64 over the CTAs in
// order, times disc): out [2d + 1].
cudaError_t launch_factor_greeks_finish(const FactorArgs &a, int grid, double disc, mc_result *out, cudaStream_t s);
size_t factor_smem_bytes(const FactorArgs &a);
cudaError_t launch_factor(const FactorArgs &a, int grid, cudaStream_t s);
int factor_occupancy(const FactorArgs &a);
int factor_paths_per_cta(const FactorArgs &a);

// Correlation sensitivities (k_corr.cu): European basket call / put,
// log-Euler, d <= kCorrMaxD; launch-parameter block with the packed FP32
// factor Lhat = log2(e) sqrt(dt) diag(sigma) Lrho (row a at a(a+1)/2), the
// per-step log2 drift and w_a S0_a (zero beyond d).
constexpr int kCorrMaxD = 64;
struct CorrConst {
    float L[kCorrMaxD * (kCorrMaxD + 1) / 2];
    float drift[kCorrMaxD];
    float ws0[kCorrMaxD];
};
struct CorrArgs {
    PathRun run;
    int d;
    int exact4;         // d % 4 == 0: every step is d/4 whole Philox blocks
    int kind;           // MC_CALL or MC_PUT on U = sum_a w_a S_a(T); MC_ASIAN_CALL or
                        // MC_ASIAN_PUT on the average of U over the steps (d <= 64)
    float strike;
    float *partials;    // [grid][64 x 64] per-CTA sums of u_a W_b (FP32)
    double *counts;     // [grid] paths simulated by each CTA
    ReduceArgs red;     // the price (one payoff)
};
int corr_occupancy(const CorrArgs &a);
int corr_block();
size_t corr_adjoint_smem(int d);
// Path kernel, batch sums (Hb [B][64 x 64], nb [B]), the Cholesky adjoint per
// batch and for all paths (out_dl, out_drho [B + 1][d x d]), and the means
// with batch-means standard errors (res_dl, res_drho [d x d]).  L: FP64
// Cholesky factor of corr [d x d]; cfac[a] = disc sqrt(dt) sigma_a.
cudaError_t launch_corr(const CorrArgs &a, const CorrConst &c, int grid, int batches, const double *L,
                        const double *cfac, double *Hb, double *nb, double *out_dl, double *out_drho,
                        mc_result *res_dl, mc_result *res_drho, cudaStream_t s);

// FP32 products (k_mlp.cu): C [M x N] = A [M x K] B^T (B stored N x K), and
// the K-slice partials part[z] [M x N] = A_z^T B_z of C = A^T B (A stored
// K x M, B stored K x N), slice z covering k in [z kchunk, (z + 1) kchunk),
// kchunk a multiple of 16.
cudaError_t gemm_f32_abt(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                         cudaStream_t s);
cudaError_t gemm_f32_atb_slices(int M, int N, int K, const float *A, int lda, const float *B, int ldb, int kchunk,
                                float *part, cudaStream_t s);

// Correlation sensitivities of wide baskets (kCorrMaxD < d <= kBigMaxD):
// W (the paths' summed normal vectors) by one kernel, Y = W Lhat^T by an
// FP32 product, the payoff slope u per path, the per-batch sums
// H_b = sum u W^T as K-slice partials of one product, and the Cholesky
// adjoint of every batch in global memory.  Scratch (caller-owned, device):
// Wbuf, Ybuf [paths x d] floats; part [batches x d x d] floats; Pm, Sm,
// out_dl, out_drho [(batches + 1) x d x d] doubles.
struct CorrWide {
    const float *Ls;      // [d x d] row-major Lhat (zero above the diagonal)
    const float *drift;   // [d] per-step log2 drift
    const float *ws0;     // [d] w_a S0_a
    const double *L;      // [d x d] FP64 Cholesky factor of corr
    const double *cfac;   // [d] disc sqrt(dt) sigma_a
    const double *nb;     // [batches] paths per batch
    int batches;
    int kchunk;           // paths per batch (a multiple of 16; the last batch may hold fewer)
    float *Wbuf, *Ybuf, *part;
    double *Lt;           // [d x d] scratch: Lrho transposed
    double *Pm, *Sm, *out_dl, *out_drho;
    mc_result *res_dl, *res_drho;
};
cudaError_t launch_corr_wide(const CorrArgs &a, const CorrWide &w, int grid, cudaStream_t s);

// Records the thread-local message returned by mc_last_error(); returns code.
int set_last_error(int code, const char *msg);
// The argument checks of mc_price (model, simulation configuration, payoff
// list), shared by every pricing entry point; fills *ps on success and sets
// the thread-local error message otherwise.
int check_price_args(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *p, int np, PayoffSet *ps);
// Polls of a bounded mbarrier wait before a tensor-core kernel gives up.
uint32_t mbar_wait_cap();

// Host launchers (return cudaError_t of the launch).
cudaError_t launch_gbm1d(const Gbm1dArgs &a, int grid, int block, cudaStream_t s);
int gbm1d_occupancy(const Gbm1dArgs &a, int block);

cudaError_t launch_basket_fp32(int D, const BasketArgs &a, const void *cst, int grid, int block,
                               cudaStream_t s);
int basket_fp32_occupancy(int D, const BasketArgs &a, int block);
int basket_fp32_width(int d);        // smallest instantiated D >= d (0 if none)
size_t basket_const_bytes(int D);    // sizeof(BasketConst<D>)
void basket_const_offsets(int D, size_t *L, size_t *drift, size_t *ws0, size_t *w, size_t *s0);

cudaError_t launch_heston(const HestonArgs &a, int grid, int block, cudaStream_t s);
int heston_occupancy(const HestonArgs &a, int block);

// Tensor-core basket: launch, occupancy, dynamic shared memory, factor prep.
cudaError_t launch_basket_tc(int prec, const TcArgs &a, const TcConst &c, int grid, cudaStream_t s);
int basket_tc_occupancy(int prec, const TcArgs &a);
// Quantised, swizzled factor image (bimg), per-column cs and drift (device).
cudaError_t launch_tc_prep(int prec, int d, const double *L, const double *sigma, double c, double sdt,
                           double r, double dt, int scheme, uint8_t *bimg, float *cs, float *drift,
                           cudaStream_t s);
int tc_bimg_bytes(int prec);

// FP64 Cholesky of a d x d SPD matrix on the device (one CTA); writes the
// lower factor to L and 0 / 1 (not positive definite) to *status.
cudaError_t launch_cholesky(int d, const double *A, double *L, int *status, cudaStream_t s);

// Lhat (packed lower triangle, FP32) = c sqrt(dt) diag(sigma) L, plus drift.
cudaError_t launch_scale_factor(int d, const double *L, const double *sigma, double c, double sdt,
                                double r, double dt, int scheme, float *Lpacked, float *drift,
                                cudaStream_t s);

}  // namespace gbmc
