/*
 * gbmc -- GB300-native financial Monte Carlo (C ABI).
 *
 * The library simulates many independent discretised SDE paths (Eq. 1 of
 * Belletti et al., "Tensor Processing Units for Financial Monte Carlo", 2019),
 * evaluates path payoffs and returns the Monte Carlo estimator of Eq. 3 with
 * its standard error.  All simulation work runs in the library's CUDA kernels
 * on the device that is current on the calling thread.
 *
 * Conventions shared by every entry point
 *   - Host pointers are read during the call only; the library copies what it
 *     needs and never frees caller memory.  Device pointers are caller-owned.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Entry
 *     points that return host results synchronise that stream before
 *     returning; mc_plan_execute is asynchronous.
 *   - Every entry point returns an mc_status.  On error no output is written,
 *     and mc_last_error() returns a thread-local message.  No entry point
 *     throws, aborts or exits.
 *   - Random numbers: Philox4x32-10 (Sec. IV.A), key = (seed mod 2^32,
 *     seed div 2^32).  Normal j of path n (global index, path_offset included)
 *     comes from the block at counter (j/4 mod 2^32, j/4 div 2^32, n mod 2^32,
 *     n div 2^32), lane j mod 4, with Box-Muller (Sec. VI.D) on lanes (0,1)
 *     and (2,3) and uniforms u(x) = (floor(x/2^9) + 1/2) 2^-23.  Step i of a
 *     d-asset GBM uses normals i*d .. i*d+d-1; step i of Heston uses 2i (the
 *     variance shock) and 2i+1.  Results therefore do not depend on the launch
 *     shape, and disjoint path_offset ranges give independent sub-runs.
 */
#ifndef GBMC_MC_H
#define GBMC_MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_VERSION 10000 /* major*10000 + minor*100 + patch */

typedef enum {
    MC_OK = 0,
    MC_EINVAL = -1,        /* an argument is out of range or inconsistent */
    MC_ENOTPSD = -2,       /* the correlation matrix is not positive definite: a pivot of
                              its FP64 Cholesky factorisation is at or below 4 d 2^-52 times
                              its diagonal entry (rank-deficient or numerically singular) */
    MC_ENOMEM = -3,        /* device or host allocation failed */
    MC_ECUDA = -4,         /* a CUDA runtime call failed (message has the name) */
    MC_ETIMEOUT = -5,      /* a bounded device wait ran out */
    MC_EUNSUPPORTED = -6   /* valid request the library does not serve */
} mc_status;

typedef enum {
    MC_GBM = 0,    /* d >= 1 correlated geometric Brownian motions (Sec. II.A.1, II.A.2) */
    MC_HESTON = 1  /* single-asset Heston stochastic volatility, full-truncation Euler */
} mc_model_kind;

typedef enum {
    MC_LOG_EULER = 0, /* Euler step on log S: exact in law at the grid for GBM */
    MC_EULER = 1      /* Euler-Maruyama step on S itself, as written in Sec. II.A.1 */
} mc_scheme;

/* Arithmetic of the correlation contraction dW = sqrt(dt) diag(sigma) L z
 * (Sec. II.A.2, Sec. V.A).  The state, the payoffs and all accumulators stay
 * FP32 whatever this is; FP64 is used only in the final cross-block sum and in
 * the Cholesky factorisation. */
typedef enum {
    MC_FP32 = 0,
    MC_BF16 = 1,     /* tensor cores, bf16 operands, FP32 accumulation */
    MC_FP16 = 2,     /* tensor cores, fp16 operands, FP32 accumulation */
    MC_FP8E4M3 = 3   /* tensor cores, e4m3 operands with per-step scale, FP32 accumulation */
} mc_precision;

typedef struct {
    int32_t kind;          /* mc_model_kind */
    int32_t d;             /* assets; MC_HESTON requires d == 1 */
    const double *s0;      /* host [d] spot prices, > 0 */
    const double *sigma;   /* host [d] volatilities >= 0 (MC_GBM) */
    const double *corr;    /* host [d*d] row-major correlation matrix (unit diagonal,
                              symmetric, positive definite), or NULL for identity */
    const double *weights; /* host [d] basket weights, or NULL for 1/d each */
    double r;              /* risk-free rate: drift of every asset and discount rate */
    double v0, kappa, theta, xi, rho; /* MC_HESTON only: dv = kappa (theta - v) dt + xi sqrt(v) dW1,
                                         d<W1, W2> = rho dt, |rho| < 1 */
    /* Factor-model correlation (MC_GBM, corr must be NULL): rho = B B^T +
     * diag(e^2), B = loadings (host [d][n_factors] row-major, every row norm
     * <= 1), e_a = sqrt(1 - sum_j B_aj^2).  Step i of path n then draws
     * normals i (k + d) + j (j < k, common factors z) and i (k + d) + k + a
     * (idiosyncratic eps_a) and uses dW_a = sqrt(dt) sigma_a (sum_j B_aj z_j
     * + e_a eps_a): O(d k) per step instead of the Cholesky O(d^2), exact in
     * law.  d <= 512, n_factors <= 16, FP32, European / Asian / barrier
     * payoffs; no Greeks, paths, two-level or QMC runs.  loadings NULL: the
     * Cholesky scheme. */
    int32_t n_factors;
    const double *loadings;
} mc_model;

/* Barrier monitoring.  MC_DISCRETE: the barrier is checked at t_1..t_M.
 * MC_BRIDGE: continuous monitoring through the maximum (minimum) of the
 * Brownian bridge between consecutive grid values x, y of log S (Sec. VI.A.1,
 * the "In and Out Put" experiment): m = (x + y + sqrt((x - y)^2 - 2 dt
 * sigma^2 ln U)) / 2 (minimum: minus the root), U uniform on (0, 1).  Single
 * asset GBM with MC_LOG_EULER only (MC_EUNSUPPORTED otherwise); the uniforms
 * are numbers 2i (maximum) and 2i + 1 (minimum) of stream 2^56 + n, the bridge
 * domain of path n, step i, mapped by the same uniform map as the normals. */
typedef enum {
    MC_DISCRETE = 0,
    MC_BRIDGE = 1
} mc_monitoring;

typedef struct {
    int32_t scheme;        /* mc_scheme (MC_GBM); MC_HESTON always uses full-truncation Euler */
    int32_t steps;         /* M >= 1 equal steps of dt = T / M */
    double T;              /* maturity > 0 */
    int64_t paths;         /* N >= 1 */
    int64_t path_offset;   /* global index of the first path (for sharding / resume) */
    uint64_t seed;         /* Philox key */
    int32_t precision;     /* mc_precision of the correlation contraction */
    int32_t ckpt_every;    /* adjoint checkpoint stride in steps (0 = 32) */
    int32_t monitoring;    /* mc_monitoring of the barrier payoffs */
} mc_sim_cfg;

/* Payoffs on the monitored underlying U(t) = sum_a w_a S_a(t) (U = S for d = 1),
 * observed at t_i = i T / M, i = 1..M (Sec. I.A.2).  Barrier kinds: up-and-out
 * is knocked out when max_i U(t_i) >= barrier, down-and-out when
 * min_i U(t_i) <= barrier; "in" kinds are alive exactly when the matching
 * "out" kind is dead.  Asian kinds use (1/M) sum_{i=1..M} U(t_i). */
typedef enum {
    MC_CALL = 0, MC_PUT = 1, MC_ASIAN_CALL = 2, MC_ASIAN_PUT = 3,
    MC_UO_CALL = 4, MC_UI_CALL = 5, MC_UO_PUT = 6, MC_UI_PUT = 7,
    MC_DO_CALL = 8, MC_DI_CALL = 9, MC_DO_PUT = 10, MC_DI_PUT = 11
} mc_payoff_kind;

#define MC_MAX_PAYOFFS 32

typedef struct {
    int32_t kind;          /* mc_payoff_kind */
    double strike;
    double barrier;        /* ignored by non-barrier kinds */
} mc_payoff;

typedef struct {
    double price;          /* e^{-rT} (1/N) sum_n f(path n): the estimator of Eq. 3 */
    double se;             /* its standard error sqrt((mean(f^2) - mean(f)^2) / (N - 1)), discounted */
} mc_result;

/* Library version (MC_VERSION of the build). */
int mc_version(void);

/* Device scratch of the set-up paths (model copies, Cholesky factors,
 * per-block partials, checkpoints) is taken from a per-device cache of blocks
 * that earlier calls released, so repeated calls of one shape allocate
 * nothing; a block is cached only once the call or plan that used it has
 * synchronised.  mc_release_cache frees every cached block (all devices) back
 * to CUDA; blocks held by live plans or running calls are not affected.
 * Returns MC_OK. */
int mc_release_cache(void);

/* Thread-local message describing the last error on this thread ("" if none). */
const char *mc_last_error(void);

/*
 * mc_debug_status -- the bounds checks of a debug build (compiled with
 * GBMC_DEBUG).  In that build the kernels check the index of their accesses
 * to caller buffers and checkpoints (materialised paths, Heston adjoint
 * checkpoints, network outputs, random-stream outputs, training labels)
 * against the buffer's extent; an access outside is skipped and recorded
 * (no trap: the kernel and the context carry on).  This call synchronises
 * the device, returns the number of skipped accesses since the previous
 * call, the site code and index of the first one (0 and 0 if none), and
 * clears them.  Site codes: 1 1-D GBM paths, 2 basket paths, 3 Heston paths,
 * 4 / 5 checkpoint store / load, 6 network output, 7 Philox words,
 * 8 normals, 9 labels.  A release build returns MC_EUNSUPPORTED.
 */
int mc_debug_status(uint32_t *violations, uint32_t *first_site, int64_t *first_index);

/*
 * The random stream (Sec. IV.A: keyed counter-based Philox4x32-10; Sec. VI.D:
 * Box-Muller), written out by the device functions every path kernel draws
 * from, e.g. to check them bit for bit against another implementation or to
 * feed the same normals to other code.  Key = (seed mod 2^32, seed div 2^32).
 *   mc_philox_words: dev_out (DEVICE, 16-byte aligned, caller-owned) [blocks][4]
 *     uint32 = Philox4x32-10 of counter (q mod 2^32, q div 2^32, n mod 2^32,
 *     n div 2^32) for q = q0 .. q0 + blocks - 1, n = stream_index.
 *     0 <= blocks <= 2^40 and the block range must not wrap past 2^64
 *     (MC_EINVAL otherwise).
 *   mc_normals: dev_out (DEVICE, caller-owned) [count] float32 = normals
 *     j0 .. j0 + count - 1 of stream stream_index (normal j from block j/4,
 *     lane j mod 4, Box-Muller on lanes (0,1) and (2,3), uniforms
 *     (floor(x/2^9) + 1/2) 2^-23; the SFU's approximate lg2, sqrt, sin and
 *     cos, so each normal is within a few 1e-6 of its exact value).
 *     0 <= count <= 2^40, no wrap past 2^64.
 * Both are asynchronous on `stream`.
 */
int mc_philox_words(uint64_t seed, uint64_t stream_index, uint64_t q0, int64_t blocks, uint32_t *dev_out,
                    void *stream);
int mc_normals(uint64_t seed, uint64_t stream_index, uint64_t j0, int64_t count, float *dev_out, void *stream);

/*
 * mc_simulate -- materialise simulated paths (Sec. II.A.1 / II.A.2 scheme).
 *   dev_out: caller-owned DEVICE buffer of float32, layout
 *            [steps/save_every + 1][D][paths], D = d for MC_GBM (asset prices)
 *            and D = 2 for MC_HESTON (price, variance before truncation);
 *            slot k holds the state after k*save_every steps (slot 0 = t_0).
 *   save_every must divide steps.  Runs on `stream` and synchronises it
 *   before returning.
 */
int mc_simulate(const mc_model *model, const mc_sim_cfg *cfg, int32_t save_every,
                float *dev_out, void *stream);

/*
 * mc_price -- discounted Monte Carlo prices of n_payoff payoffs on the same
 * simulated paths (Eq. 3), with standard errors.
 *   out: host [n_payoff] results.  1 <= n_payoff <= MC_MAX_PAYOFFS.
 * Synchronises `stream` before returning.
 */
int mc_price(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs,
             int32_t n_payoff, mc_result *out, void *stream);

/*
 * mc_greek_count -- number of Greeks mc_greeks returns per payoff:
 *   MC_GBM: 2d + 1 (d/dS0_a, a < d; d/dsigma_a; d/dr), MC_HESTON: 7
 *   (d/dS0, d/dv0, d/dr, d/dkappa, d/dtheta, d/dxi, d/drho).  -1 on NULL.
 */
int32_t mc_greek_count(const mc_model *model);

/*
 * mc_greeks -- pathwise (infinitesimal perturbation) Greeks of the discounted
 * prices (Sec. I.A.3; the paper obtains them by back-propagation through the
 * simulation, Sec. VI.A.2), with their standard errors, on the same paths as
 * the prices.  d/dr includes the -T * price term of the discount factor.
 *   MC_HESTON: reverse-mode adjoint kernel; the path state is checkpointed
 *     every cfg->ckpt_every steps (0 = 32, at most 64) in device scratch and
 *     each segment is recomputed from its checkpoint during the backward
 *     sweep.  d sqrt(v+)/dv is taken as 0 where v <= 0.
 *   MC_GBM, d == 1: MC_LOG_EULER (the adjoint of log S is constant along
 *     the path and the sweep reduces to closed forms per path); European and
 *     Asian payoffs, 1 <= n_payoff.
 *   MC_GBM, 2 <= d <= 512 (correlated basket on U = sum_a w_a S_a): exactly
 *     one payoff, MC_CALL or MC_PUT on U(T) (MC_EINVAL for n_payoff != 1,
 *     MC_EUNSUPPORTED for other kinds); MC_LOG_EULER; sigma_a > 0 for every
 *     asset (MC_EINVAL otherwise); any cfg->precision (the Greeks' per-path
 *     terms are formed in the path kernel's epilogue from the same paths as
 *     the price).  greeks[0..d-1] = delta_a = dP/dS0_a,
 *     greeks[d..2d-1] = vega_a = dP/dsigma_a (sigma_a scales column a of
 *     diag(sigma) Lrho), greeks[2d] = rho = dP/dr.  MC_ENOTPSD if corr is
 *     not positive definite, MC_ETIMEOUT if a bounded device wait gave up.
 *   MC_GBM with loadings (the factor model): the same layout and payoff
 *     rules, MC_LOG_EULER and MC_FP32; sigma_a scales asset a's whole
 *     increment (loadings and idiosyncratic weight held fixed), so
 *     vega_a = e^{-rT} E[f' w_a S_a (ln(S_a/S0_a) - (r + sigma_a^2/2) T) / sigma_a].
 * Barrier payoffs are rejected (a knock indicator has no pathwise derivative:
 * MC_EUNSUPPORTED).
 *   prices: host [n_payoff] or NULL; greeks: host [n_payoff][mc_greek_count].
 * Synchronises `stream` before returning.
 */
int mc_greeks(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs, int32_t n_payoff,
              mc_result *prices, mc_result *greeks, void *stream);

/*
 * mc_corr_greeks -- pathwise sensitivities of a European basket call or put
 * on U = sum_a w_a S_a(T), or (d <= 64) of an Asian one (MC_ASIAN_CALL /
 * MC_ASIAN_PUT: on the average of U over the steps), to the correlation
 * matrix (Sec. I.A.3:
 * sensitivities to model parameters; Sec. II.A.2: dW = sqrt(dt) diag(sigma)
 * Lrho z with Lrho the Cholesky factor of corr; Sec. VI.A.2 differentiates
 * the basket simulation), reverse mode, FP32 paths and FP64 post-processing.
 *   model: MC_GBM, 2 <= d <= 512, corr given or NULL (= identity), no
 *          loadings.  cfg: MC_LOG_EULER, MC_FP32, MC_DISCRETE.  For d > 64
 *          the per-path vectors live in device scratch (8 d bytes per path;
 *          paths x d <= 2^31) and the path contractions run as FP32
 *          products.
 *   payoff: one MC_CALL or MC_PUT, or for d <= 64 MC_ASIAN_CALL or
 *          MC_ASIAN_PUT (weights from the model, 1/d if NULL).  The Asian
 *          form runs every path twice: once to its average and payoff slope,
 *          then again adding the slope-weighted outer products of every
 *          step.
 *   price: host [1] or NULL: the discounted price and its standard error.
 *   dl:    host [d*d] or NULL, row-major: dP/dLrho[a][b] for b <= a (the
 *          entry's coefficient in dW_a, the drift (r - sigma_a^2/2) held
 *          fixed); zero above the diagonal.
 *   drho:  host [d*d] or NULL, row-major: dP/dcorr[a][b] for a != b, with
 *          corr[a][b] and corr[b][a] moved together (symmetric); zero on the
 *          diagonal.
 * Standard errors of dl and drho are batch-means errors over min(64, CTAs of
 * the launch) groups of paths for d <= 64, min(32, ceil(paths / 128))
 * contiguous groups for d > 64 (NaN with one group, i.e. paths <= 128); the
 * price's is the usual one.  Errors: MC_EUNSUPPORTED outside the cases above,
 * MC_ENOTPSD if corr is not positive definite, MC_EINVAL on bad arguments;
 * outputs are untouched on error.  Synchronises `stream` before returning.
 */
int mc_corr_greeks(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoff, mc_result *price,
                   mc_result *dl, mc_result *drho, void *stream);

/*
 * mc_price_mlmc -- two-level precision estimator (Sec. V: a fast reduced-
 * precision simulation whose bias is identified with few samples and
 * corrected; Giles' multilevel Monte Carlo over precisions):
 *   price = mean_{N0}(P_q) + mean_{N1}(P_fp32 - P_q),
 * level 0 = the tensor-core kernel with cfg->precision (BF16, FP16 or E4M3)
 * on paths [path_offset, path_offset + cfg->paths); level 1 = paths_ref
 * further paths [path_offset + cfg->paths, ... + paths_ref), each simulated
 * twice on the same normals: the FP32 contraction, and the tensor-core
 * operand rounding with FP32 accumulation.  The two levels use disjoint
 * paths, so se^2 = se_0^2 + se_1^2.
 *   Correlated GBM baskets with 2 <= d <= 64, discrete monitoring;
 *   1 <= n_payoff <= 10; paths_ref >= 2.  out: host [n_payoff].
 * Errors: MC_EINVAL for bad arguments (an FP32 cfg->precision, counts
 * outside the limits), MC_EUNSUPPORTED outside the cases above, MC_ENOTPSD
 * if corr is not positive definite, MC_ETIMEOUT if a bounded wait of the
 * tensor-core level expires; out is untouched on error.  Synchronises
 * `stream`.
 */
typedef struct {
    double price, se;         /* the two-level estimate of the FP32 price */
    mc_result coarse;         /* level 0: reduced precision, cfg->paths paths */
    mc_result correction;     /* level 1: mean of P_fp32 - P_q, paths_ref paths */
    mc_result ref_level;      /* level 1's P_fp32 alone */
    mc_result coarse_level;   /* level 1's P_q alone */
} mc_mlmc_result;
int mc_price_mlmc(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs, int32_t n_payoff,
                  int64_t paths_ref, mc_mlmc_result *out, void *stream);

/*
 * mc_price_qmc -- randomised quasi-Monte Carlo (Sec. IV, Sobol QRNGs; the
 * basket experiment of Sec. VI.D): the GBM basket of `model` driven by a
 * Sobol sequence instead of Philox normals.  Dimension 1 is van der Corput;
 * dimension j >= 2 uses the (j-1)-th primitive polynomial over GF(2) (by
 * degree, then value) with initial direction integers m_1..m_s = 1 and the
 * Bratley-Fox recurrence.  Point n of dimension j is the XOR of the direction
 * words over the set bits of n; replication r XORs dimension j with word j of
 * Philox stream 6 * 2^56 + r under cfg->seed (a random digital shift).
 * Normal a of step i is the cosine branch of Box-Muller on dimensions
 * 2 (i d + a), 2 (i d + a) + 1, through the uniform map of the Philox path.
 *   cfg->paths = points per replication, cfg->path_offset = first point;
 *   points in [0, 2^23); d <= 32 and 2 d steps <= 64; FP32 contraction,
 *   discrete monitoring; 2 <= replications <= 65535.
 *   out: host [n_payoff]: price = mean of the replication means, se = their
 *   standard deviation / sqrt(replications).  rep_means: optional host
 *   [replications][n_payoff].
 * Errors: MC_EINVAL for bad arguments (replications or the point range out
 * of bounds), MC_EUNSUPPORTED outside the cases above (d, dimensions,
 * precision), MC_ENOTPSD if corr is not positive definite; outputs are
 * untouched on error.  Synchronises `stream`.
 */
int mc_price_qmc(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs, int32_t n_payoff,
                 int32_t replications, mc_result *out, double *rep_means, void *stream);

/*
 * Surrogate pricing network (mc_mlp): n_in -> width x hidden (SiLU) -> 1
 * (linear), the network that revalues the risk portfolio (Sec. VI.B; its
 * layers are the DNN layer / simulation time step analogy of Sec. III.C,
 * trained by back-propagation, Sec. I.A.3).  Parameters are
 * one packed FP32 vector: for each layer l, W_l [in x out] row-major, then
 * b_l [out].  All x / y / t buffers are DEVICE pointers, row-major [n x n_in]
 * and [n]; host pointers are noted.  The network lives on the device that
 * was current at creation.
 *   mc_mlp_create: init = host packed parameters (mc_mlp_param_count floats).
 *   mc_mlp_forward: y = net(x); precision MC_FP32 (FP32 SIMT GEMMs) or
 *     MC_BF16 (tensor cores, BF16 weights and activations, FP32 accumulation).
 *   mc_mlp_loss_grad: MSE (1/n) sum (y - t)^2 and its gradient (host, packed;
 *     may be NULL) by back-propagation; synchronises `stream`.
 *   mc_mlp_train: `epochs` passes of mini-batch Adam (lr; beta 0.9, 0.999;
 *     eps 1e-8) over the n samples in whole batches; last_epoch_loss = mean
 *     batch loss of the final epoch; synchronises `stream`.
 *   mc_mlp_set_train_mode: arithmetic of mc_mlp_loss_grad and mc_mlp_train.
 *     MC_MLP_TRAIN_FP32 (default): FP32 SIMT products.  MC_MLP_TRAIN_TF32X3:
 *     the width -> width layers' forward, input-gradient and weight-gradient
 *     products on the tensor cores with operands split hi + lo and
 *     accumulated as hi*hi + hi*lo + lo*hi in FP32 (FP32-like accuracy); needs
 *     >= 2 hidden layers of a width that is a multiple of 64
 *     (MC_EUNSUPPORTED otherwise).  It also selects the arithmetic of
 *     mc_mlp_loss_grad_d, mc_mlp_train_d and mc_mlp_loss_grad_sums.  A
 *     bounded wait that expires makes the call return MC_ETIMEOUT.
 * Errors: MC_EINVAL for a NULL network or buffer, n < 1, sizes outside the
 * limits above, or a learning rate that is not > 0 (checked before any
 * device work); MC_ECUDA when a CUDA call fails.  The caller owns every buffer; the
 * network owns its parameters and Adam state until mc_mlp_destroy.
 */
#define MC_MLP_TRAIN_FP32 0
#define MC_MLP_TRAIN_TF32X3 1
typedef struct mc_mlp mc_mlp;
int mc_mlp_create(int32_t n_in, int32_t width, int32_t hidden, const float *init, mc_mlp **net);
int64_t mc_mlp_param_count(const mc_mlp *net);
int mc_mlp_get_params(const mc_mlp *net, float *host);
int mc_mlp_set_params(mc_mlp *net, const float *host);
int mc_mlp_forward(mc_mlp *net, const float *dev_x, int64_t n, float *dev_y, int32_t precision, void *stream);
int mc_mlp_loss_grad(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, double *loss,
                     float *host_grad, void *stream);
int mc_mlp_train(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, int32_t epochs, int32_t batch,
                 float lr, double *last_epoch_loss, void *stream);
/* One Adam step (the update of mc_mlp_train) with a given gradient: host_grad
 * [mc_mlp_param_count] host floats, e.g. the average of the ranks' batch
 * gradients in data-parallel training.  Synchronises `stream`. */
int mc_mlp_apply_grad(mc_mlp *net, const float *host_grad, float lr, void *stream);
/*
 * Training on prices and their sensitivities (derivative labels; the
 * network is fitted to the Monte Carlo prices and to their pathwise Greeks,
 * Sec. I.A.3): the loss is
 *   (1/n) sum_i [(y_i - t_i)^2 + sum_k weight_k m_ik (scale_k dy_i/dx_{dir_k} - g_ik)^2],
 * m_ik = 1 where g_ik is finite, 0 where it is not (a sample without that
 * label, e.g. a barrier point's NaN from mc_surrogate_label_greeks).  dy/dx is
 * the network's input gradient (forward-mode tangents through the layers) and
 * the loss is differentiated through it (a reverse sweep through the
 * tangents, with the activation's second derivative).  FP32 SIMT products,
 * or, in MC_MLP_TRAIN_TF32X3, the width -> width products of the stacked
 * primal and tangent rows on the tensor cores as in mc_mlp_loss_grad; the
 * network needs a hidden layer.
 *   dl: n_dir in [0, 4] directions; dir[k] an input index, scale[k] finite
 *     (scale_k = 1 / (the input map's slope) turns a network-input derivative
 *     into a derivative in the raw variable), weight[k] >= 0.
 *   dev_g: DEVICE [n][n_dir] floats (may be NULL when n_dir = 0).
 *   mc_mlp_loss_grad_d: loss_parts host [1 + n_dir] (price term, then each
 *     direction's weighted term) or NULL; host_grad as in mc_mlp_loss_grad.
 *   mc_mlp_train_d: as mc_mlp_train with this loss (last_epoch_loss = the
 *     mean total loss of the final epoch).  Both synchronise `stream`.
 */
typedef struct {
    int32_t n_dir;
    int32_t dir[4];
    float scale[4];
    float weight[4];
} mc_mlp_dloss;
int mc_mlp_loss_grad_d(mc_mlp *net, const float *dev_x, const float *dev_t, const float *dev_g, int64_t n,
                       const mc_mlp_dloss *dl, double *loss_parts, float *host_grad, void *stream);
int mc_mlp_train_d(mc_mlp *net, const float *dev_x, const float *dev_t, const float *dev_g, int64_t n,
                   const mc_mlp_dloss *dl, int32_t epochs, int32_t batch, float lr, double *last_epoch_loss,
                   void *stream);
/* Data-parallel training without host round trips (every buffer on the
 * network's device, everything asynchronous on `stream`):
 *   mc_mlp_loss_grad_sums: dev_out [count + 1] floats: [0, count) = the
 *     gradient of the batch's SUMMED loss sum_i (y_i - t_i)^2 (n times the
 *     gradient of mc_mlp_loss_grad), [count] = that summed loss; adding the
 *     ranks' buffers (an all-reduce) gives the global batch's sums.
 *   mc_mlp_apply_grad_sums: one Adam step with gradient scale * dev_grad
 *     (scale = 1 / global batch size turns summed gradients into the mean).
 * A bounded wait that expires in the tensor-core training products is
 * reported by the network's next synchronising call (MC_ETIMEOUT). */
int mc_mlp_loss_grad_sums(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, float *dev_out,
                          void *stream);
int mc_mlp_apply_grad_sums(mc_mlp *net, const float *dev_grad, float scale, float lr, void *stream);
int mc_mlp_set_train_mode(mc_mlp *net, int32_t mode);
int mc_mlp_destroy(mc_mlp *net);

/*
 * Portfolio risk (Sec. VI.B): VaR and CVaR of the one-period PnL of a
 * portfolio of options on correlated GBM underlyings.
 *   Scenarios: S'_u = S0_u exp((mu - sigma_u^2/2) h + sqrt(h) sigma_u (Lrho z)_u),
 *   z = normals of scenario stream s (a stream domain of its own).
 *   Revaluation of every option at (S', T_o - h): MC_RISK_NESTED runs
 *   inner_paths Monte Carlo paths per (scenario, underlying) with steps of
 *   1 / steps_per_year (up-and-out calls monitored at every step, and
 *   worthless when S' is already at or above the barrier); base values at
 *   (S0, T_o) use base_paths paths.  MC_RISK_SURROGATE evaluates the network
 *   v = V_call / K at the inputs of (S/K, sigma, tau, r, K/H) (K/H = 0 for
 *   European; inputs as written by mc_surrogate_labels), puts by put-call
 *   parity, at the scenario states and at the base date.
 *   PnL_s = sum_o position_o (V_o(scenario s) - V_o(base)); losses l = -PnL;
 *   VaR_alpha = the k-th largest loss, k = ceil((1 - alpha) n_scen);
 *   CVaR_alpha = the mean of the losses strictly above VaR_alpha (VaR_alpha
 *   itself if none is).  Maturities and the horizon are whole steps.
 *   Limits: n_under <= 64, 32 options per underlying, n_scen <= 2^24;
 *   option kinds MC_CALL, MC_PUT, MC_UO_CALL.
 *   host_pnl: host [n_scen] or NULL.  Synchronises `stream`.
 * Errors (checked before any device work unless noted): MC_EINVAL for NULL
 * arrays, counts or limits outside the above, non-positive s0 or strike,
 * negative sigma, maturities or a horizon that are not whole steps, a
 * missing surrogate or one without 5 inputs; MC_EUNSUPPORTED for another
 * option kind; MC_ENOTPSD when corr is not positive definite (after the
 * device Cholesky); MC_ETIMEOUT when a bounded wait of the surrogate's
 * kernel expired.  res and host_pnl are untouched on error.
 */
typedef struct {
    int32_t n_under;
    const double *s0, *sigma, *corr; /* [n_under], [n_under], [n_under^2] or NULL */
    double r;                        /* risk-free rate (revaluation, discounting) */
    double mu;                       /* drift of the scenario move */
    int32_t n_opt;
    const int32_t *under;            /* [n_opt] underlying index */
    const int32_t *kind;             /* [n_opt] MC_CALL, MC_PUT or MC_UO_CALL */
    const double *strike, *barrier, *maturity, *position; /* [n_opt]; barrier may be NULL without barriers */
} mc_portfolio;

typedef enum { MC_RISK_NESTED = 0, MC_RISK_SURROGATE = 1 } mc_risk_method;

typedef struct {
    double alpha;            /* e.g. 0.99 */
    double horizon;          /* h in years, a whole number of steps */
    int64_t n_scen;
    int32_t steps_per_year;  /* time step of the revaluation, e.g. 252 (daily) */
    int32_t method;          /* mc_risk_method */
    int32_t inner_paths;     /* nested: paths per (scenario, underlying) */
    int32_t base_paths;      /* nested: paths per underlying at the base date */
    uint64_t seed;
    mc_mlp *surrogate;       /* surrogate: the trained network */
    int32_t surrogate_precision; /* MC_FP32 or MC_BF16 */
    int64_t scen_offset;     /* global index of the first scenario: a run over
                                [scen_offset, scen_offset + n_scen) reproduces that
                                slice of a run from 0 (sharding across devices);
                                VaR / CVaR are those of this slice */
} mc_risk_cfg;

typedef struct {
    double var, cvar;        /* of the loss -PnL */
    double base_value;       /* sum_o position_o V_o(base) */
    int64_t n_tail;          /* losses strictly above VaR */
} mc_risk_result;

int mc_risk(const mc_portfolio *portfolio, const mc_risk_cfg *cfg, mc_risk_result *result, double *host_pnl,
            void *stream);

/*
 * mc_tail -- VaR and CVaR (Sec. VI.B, the selection of mc_risk) of the
 * losses -pnl over a DEVICE vector of n PnLs, e.g. every shard's scenario
 * PnLs gathered on one device: VaR_alpha = the k-th largest loss,
 * k = ceil((1 - alpha) n); CVaR_alpha = the mean of the losses strictly above
 * VaR_alpha (VaR_alpha itself if none is); n_tail = their count;
 * base_value = 0.  1 <= n <= 2^24, 0 < alpha < 1.  Synchronises `stream`.
 */
int mc_tail(const double *dev_pnl, int64_t n, double alpha, mc_risk_result *result, void *stream);

/*
 * mc_surrogate_labels -- training set of the surrogate: for each point p of
 * dev_points [n][5] = (S/K, sigma, tau, r, K/H), the label dev_labels[p] =
 * discounted Monte Carlo price / K of a call on S with strike K and maturity
 * tau (an up-and-out call with barrier H monitored at every step when
 * K/H > 0; 0 when S >= H), with `paths` paths and round(tau * steps_per_year)
 * log-Euler steps on a stream domain of its own; and, if dev_inputs is not
 * NULL, the network inputs dev_inputs [n][5] =
 *   ((S/K - 1.05)/0.55, (sigma - 0.25)/0.15, tau - 1, (r - 0.04)/0.04,
 *    (K/H - 0.45)/0.45),
 * the same map mc_risk applies before evaluating the network.  Asynchronous
 * on `stream`.
 */
int mc_surrogate_labels(int64_t n_points, const float *dev_points, int32_t paths, int32_t steps_per_year,
                        uint64_t seed, float *dev_labels, float *dev_inputs, void *stream);
/*
 * mc_surrogate_label_greeks -- mc_surrogate_labels (same paths, same labels)
 * plus the pathwise sensitivities of each label (Sec. I.A.3): dev_dlabels
 * DEVICE [n][2] = (d label / d(S/K), d label / d sigma), i.e. the discounted
 * path means of 1{S_T > K} S_T / S and 1{S_T > K} (S_T / K)
 * (sqrt(dt) sum_i z_i - sigma tau).  Barrier points (K/H > 0) get NaN: a
 * knock-out indicator has no pathwise derivative.  dev_inputs as in
 * mc_surrogate_labels (may be NULL).  Asynchronous on `stream`.
 */
int mc_surrogate_label_greeks(int64_t n_points, const float *dev_points, int32_t paths, int32_t steps_per_year,
                              uint64_t seed, float *dev_labels, float *dev_dlabels, float *dev_inputs, void *stream);

/*
 * Plans: the same computation as mc_price (the paths of Eq. 1, the estimator
 * of Eq. 3) split into a set-up phase (argument
 * checks, upload of the model, FP64 Cholesky factorisation on the device,
 * scaled copies of the factor, device scratch for per-block partial sums)
 * and an asynchronous execution that launches only the path kernels and the
 * final FP64 reduction.  A plan may be executed any number of times on any
 * stream of the device it was created on, but executions of one plan must
 * not overlap in time (they share the plan's scratch).
 *   mc_plan_execute: dev_out is a DEVICE buffer of n_payoff mc_result.
 * Errors: mc_plan_create returns mc_price's argument errors (MC_EINVAL,
 * MC_EUNSUPPORTED, MC_ENOTPSD) before launching anything; mc_plan_execute
 * returns MC_EINVAL for a NULL plan or buffer and MC_ECUDA when a launch
 * fails.  The plan owns its device scratch until mc_plan_destroy.
 */
typedef struct mc_plan mc_plan;
int mc_plan_create(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs,
                   int32_t n_payoff, mc_plan **plan, void *stream);
int mc_plan_execute(mc_plan *plan, mc_result *dev_out, void *stream);
int mc_plan_destroy(mc_plan *plan);

/* Number of kernel launches one mc_plan_execute issues (for accounting). */
int mc_plan_launches(const mc_plan *plan);

/*
 * Runs over disjoint path ranges (path_offset; one per device or process)
 * combine into the estimator of Eq. 3 over their union:
 *   mc_moments: moments [n_payoff][3] = (N mean, N mean(f^2), N), discounted
 *     units, of a run's results over N = paths paths (recovered from
 *     price and se exactly up to rounding).
 *   mc_combine: out [n_payoff] = (price, se) from moments summed over runs
 *     (e.g. by an all-reduce).
 * Host arrays only; no device work.  MC_EINVAL on non-finite input.
 */
int mc_moments(const mc_result *res, int32_t n_payoff, int64_t paths, double *moments);
int mc_combine(const double *moments, int32_t n_payoff, mc_result *out);

/*
 * mc_price_gbm1d_noalloc -- single-asset GBM pricing that allocates nothing.
 * (The paper has no counterpart: this is a deployment variant of mc_price.)
 *
 * For callers that must not call cudaMalloc or any allocating routine: code
 * that runs under another framework's memory pool or allocator hooks, or
 * inside a latency-critical loop where a device allocation (which can
 * synchronise the device) is not allowed.  The caller passes the inputs
 * (host structs, as for mc_price) and the output; the kernel's scratch
 * (per-block FP32 partial sums and the last-block ticket) is a fixed device
 * array inside the library, MC_NOALLOC_PARTIALS floats (512 KiB) plus 256
 * bytes, which every GPU that loads the library holds until the process
 * exits.
 *   model: kind MC_GBM with d == 1; cfg, payoffs as for mc_price
 *          (1 <= n_payoff <= MC_MAX_PAYOFFS; larger counts are rejected with
 *          MC_EINVAL).  The grid is limited to the blocks whose partial sums
 *          fit the array; any path count is accepted.
 *   dev_out: DEVICE buffer of n_payoff mc_result, written asynchronously on
 *          `stream`; nothing is synchronised.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  Every call shares the one array and leaves its contents behind;
 * the ticket that must start at zero is cleared at each call.  Calls whose
 * executions overlap on the GPU (other streams, other threads) race on the
 * array: serialise them.
 */
#define MC_NOALLOC_PARTIALS 131072
int mc_price_gbm1d_noalloc(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs,
                           int32_t n_payoff, mc_result *dev_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBMC_MC_H */
