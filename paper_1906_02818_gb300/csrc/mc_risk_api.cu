// C ABI of portfolio risk (mc_risk) and of the surrogate's training labels
// (mc_surrogate_labels): argument checks, the option layout the kernels use
// (grouped by underlying, sorted by maturity), the FP64 Cholesky of the
// underlyings' correlation, and the sequence outer scenarios -> revaluation
// (nested Monte Carlo or the network) -> PnL -> VaR / CVaR.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <vector>

#include "mc_kernels.cuh"
#include "mlp.cuh"
#include "risk.cuh"

using namespace gbmc;

// Layout of struct mc_mlp shared with mc_mlp_api.cu (parameters and layout).
struct mc_mlp;
namespace gbmc {
const MlpLayout &mlp_layout_of(const mc_mlp *net);
int mlp_forward_any(mc_mlp *net, const float *x, int64_t n, float *y, int precision, cudaStream_t s);
int mlp_check_timeout(mc_mlp *net, cudaStream_t s);
}  // namespace gbmc

namespace {

#define RK_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            char b_[256];                                                                     \
            std::snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));           \
            return set_last_error(e_ == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA, b_); \
        }                                                                                     \
    } while (0)

int fail(int code, const char *msg) { return set_last_error(code, msg); }

struct DevBufs {
    std::vector<void *> ptrs;
    template <class T>
    cudaError_t alloc(T **p, size_t n)
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T) + 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~DevBufs()
    {
        for (void *p : ptrs) cudaFree(p);
    }
};

}  // namespace

extern "C" {

static int labels_common(int64_t n_points, const float *dev_points, int32_t paths, int32_t steps_per_year,
                         uint64_t seed, float *dev_labels, float *dev_inputs, float *dev_dlabels, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: surrogate labels");
    if (n_points < 1 || !dev_points || !dev_labels) return fail(MC_EINVAL, "points and labels must be set, n >= 1");
    if (n_points > (int64_t(1) << 36)) return fail(MC_EINVAL, "too many points");
    if (paths < 1 || paths > 65536) return fail(MC_EINVAL, "paths must lie in [1, 65536]");
    if (steps_per_year < 1) return fail(MC_EINVAL, "steps_per_year must be >= 1");
    RK_CUDA(launch_labels(n_points, dev_points, paths, static_cast<float>(steps_per_year),
                          round_keys(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)), dev_labels, dev_inputs,
                          dev_dlabels, static_cast<cudaStream_t>(stream)));
    return MC_OK;
}

int mc_surrogate_labels(int64_t n_points, const float *dev_points, int32_t paths, int32_t steps_per_year,
                        uint64_t seed, float *dev_labels, float *dev_inputs, void *stream)
{
    return labels_common(n_points, dev_points, paths, steps_per_year, seed, dev_labels, dev_inputs, nullptr, stream);
}

int mc_surrogate_label_greeks(int64_t n_points, const float *dev_points, int32_t paths, int32_t steps_per_year,
                              uint64_t seed, float *dev_labels, float *dev_dlabels, float *dev_inputs, void *stream)
{
    if (!dev_dlabels) return fail(MC_EINVAL, "dev_dlabels must be set");
    return labels_common(n_points, dev_points, paths, steps_per_year, seed, dev_labels, dev_inputs, dev_dlabels,
                         stream);
}

int mc_tail(const double *dev_pnl, int64_t n, double alpha, mc_risk_result *res, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_tail");
    if (!dev_pnl || !res) return fail(MC_EINVAL, "dev_pnl and result must be set");
    if (n < 1 || n > (int64_t(1) << 24)) return fail(MC_EINVAL, "n outside [1, 2^24]");
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(MC_EINVAL, "alpha must lie in (0, 1)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    DevBufs B;
    double *d_work, *d_res;
    RK_CUDA(B.alloc(&d_work, np2));
    RK_CUDA(B.alloc(&d_res, 3));
    RK_CUDA(launch_tail(n, dev_pnl, d_work, np2, alpha, d_res, s));
    double r3[3];
    RK_CUDA(cudaMemcpyAsync(r3, d_res, sizeof r3, cudaMemcpyDeviceToHost, s));
    RK_CUDA(cudaStreamSynchronize(s));
    res->var = r3[0];
    res->cvar = r3[1];
    res->n_tail = static_cast<int64_t>(r3[2]);
    res->base_value = 0.0;
    return MC_OK;
}

int mc_risk(const mc_portfolio *pf, const mc_risk_cfg *cf, mc_risk_result *res, double *host_pnl, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_risk");
    if (!pf || !cf || !res) return fail(MC_EINVAL, "portfolio, cfg and result must be set");
    const int d = pf->n_under, no = pf->n_opt;
    if (d < 1 || d > kRiskMaxUnder) return fail(MC_EINVAL, "n_under outside [1, 64]");
    if (no < 1 || no > d * kRiskMaxOptPerUnder) return fail(MC_EINVAL, "n_opt outside [1, 32 n_under]");
    if (!pf->s0 || !pf->sigma || !pf->under || !pf->kind || !pf->strike || !pf->maturity || !pf->position)
        return fail(MC_EINVAL, "portfolio arrays must be set");
    if (!(cf->alpha > 0.0 && cf->alpha < 1.0)) return fail(MC_EINVAL, "alpha must lie in (0, 1)");
    if (cf->n_scen < 1 || cf->n_scen > (int64_t(1) << 24)) return fail(MC_EINVAL, "n_scen outside [1, 2^24]");
    if (cf->scen_offset < 0 || cf->scen_offset + cf->n_scen > (int64_t(1) << 34))
        return fail(MC_EINVAL, "scenario range must lie in [0, 2^34)");
    if (cf->steps_per_year < 1) return fail(MC_EINVAL, "steps_per_year must be >= 1");
    const double spy = cf->steps_per_year, dt = 1.0 / spy;
    const int hsteps = static_cast<int>(std::lround(cf->horizon * spy));
    if (hsteps < 1 || std::fabs(hsteps * dt - cf->horizon) > 1e-9)
        return fail(MC_EINVAL, "horizon must be a whole number of steps");
    if (cf->method == MC_RISK_NESTED && (cf->inner_paths < 1 || cf->inner_paths > 65536 || cf->base_paths < 1 ||
                                         cf->base_paths > (1 << 24)))
        return fail(MC_EINVAL, "inner_paths in [1, 65536], base_paths in [1, 2^24]");
    if (cf->method == MC_RISK_SURROGATE && !cf->surrogate) return fail(MC_EINVAL, "surrogate network not set");
    if (cf->method != MC_RISK_NESTED && cf->method != MC_RISK_SURROGATE) return fail(MC_EINVAL, "unknown method");
    for (int u = 0; u < d; ++u)
        if (!(pf->s0[u] > 0.0) || !(pf->sigma[u] >= 0.0)) return fail(MC_EINVAL, "s0 > 0 and sigma >= 0 required");

    // option layout: grouped by underlying, sorted by maturity
    std::vector<int> order(no);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int> steps(no);
    for (int o = 0; o < no; ++o) {
        const int u = pf->under[o], k = pf->kind[o];
        if (u < 0 || u >= d) return fail(MC_EINVAL, "option underlying out of range");
        if (k != MC_CALL && k != MC_PUT && k != MC_UO_CALL) return fail(MC_EUNSUPPORTED, "risk portfolio kinds: call, put, up-and-out call");
        const long st = std::lround(pf->maturity[o] * spy);
        if (st <= hsteps || std::fabs(st * dt - pf->maturity[o]) > 1e-9)
            return fail(MC_EINVAL, "maturities must be whole steps beyond the horizon");
        if (!(pf->strike[o] > 0.0)) return fail(MC_EINVAL, "strike must be > 0");
        if (k == MC_UO_CALL && !(pf->barrier && pf->barrier[o] > 0.0)) return fail(MC_EINVAL, "barrier must be > 0");
        steps[o] = static_cast<int>(st);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return pf->under[a] != pf->under[b] ? pf->under[a] < pf->under[b] : steps[a] < steps[b];
    });
    std::vector<int> h_under(no), h_kind(no), h_rem(no), h_start(d + 1, 0);
    std::vector<float> h_K(no), h_H(no);
    std::vector<double> h_pos(no);
    for (int i = 0; i < no; ++i) {
        const int o = order[i];
        h_under[i] = pf->under[o];
        h_kind[i] = pf->kind[o];
        h_rem[i] = steps[o] - hsteps;
        h_K[i] = static_cast<float>(pf->strike[o]);
        h_H[i] = pf->kind[o] == MC_UO_CALL ? static_cast<float>(pf->barrier[o]) : INFINITY;
        h_pos[i] = pf->position[o];
        h_start[pf->under[o] + 1]++;
    }
    for (int u = 0; u < d; ++u) {
        if (h_start[u + 1] > kRiskMaxOptPerUnder) return fail(MC_EINVAL, "more than 32 options on one underlying");
        h_start[u + 1] += h_start[u];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBufs B;
    int *d_under, *d_kind, *d_rem, *d_start, *d_status;
    float *d_K, *d_H, *d_s0, *d_sig, *d_Lc, *d_drift, *d_Sp;
    double *d_pos, *d_base, *d_corr, *d_L, *d_pnl, *d_work, *d_res;
    const int64_t ns = cf->n_scen;
    int64_t np2 = 1;
    while (np2 < ns) np2 <<= 1;
    RK_CUDA(B.alloc(&d_under, no)); RK_CUDA(B.alloc(&d_kind, no)); RK_CUDA(B.alloc(&d_rem, no));
    RK_CUDA(B.alloc(&d_start, d + 1)); RK_CUDA(B.alloc(&d_status, 1));
    RK_CUDA(B.alloc(&d_K, no)); RK_CUDA(B.alloc(&d_H, no)); RK_CUDA(B.alloc(&d_s0, d)); RK_CUDA(B.alloc(&d_sig, d));
    RK_CUDA(B.alloc(&d_Lc, d * d)); RK_CUDA(B.alloc(&d_drift, d)); RK_CUDA(B.alloc(&d_Sp, ns * d));
    RK_CUDA(B.alloc(&d_pos, no)); RK_CUDA(B.alloc(&d_base, no)); RK_CUDA(B.alloc(&d_corr, d * d));
    RK_CUDA(B.alloc(&d_L, d * d)); RK_CUDA(B.alloc(&d_pnl, ns)); RK_CUDA(B.alloc(&d_work, np2)); RK_CUDA(B.alloc(&d_res, 3));
    std::vector<float> h_s0(d), h_sig(d);
    for (int u = 0; u < d; ++u) {
        h_s0[u] = static_cast<float>(pf->s0[u]);
        h_sig[u] = static_cast<float>(pf->sigma[u]);
    }
    std::vector<double> corr(static_cast<size_t>(d) * d, 0.0);
    if (pf->corr) std::copy(pf->corr, pf->corr + static_cast<size_t>(d) * d, corr.begin());
    else for (int u = 0; u < d; ++u) corr[static_cast<size_t>(u) * d + u] = 1.0;
    RK_CUDA(cudaMemcpyAsync(d_under, h_under.data(), no * sizeof(int), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_kind, h_kind.data(), no * sizeof(int), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_rem, h_rem.data(), no * sizeof(int), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_start, h_start.data(), (d + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_K, h_K.data(), no * sizeof(float), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_H, h_H.data(), no * sizeof(float), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_pos, h_pos.data(), no * sizeof(double), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_s0, h_s0.data(), d * sizeof(float), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_sig, h_sig.data(), d * sizeof(float), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_corr, corr.data(), corr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    RK_CUDA(launch_cholesky(d, d_corr, d_L, d_status, s));
    std::vector<double> L(static_cast<size_t>(d) * d);
    int status = 0;
    RK_CUDA(cudaMemcpyAsync(L.data(), d_L, L.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RK_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    RK_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    const double h = hsteps * dt;
    std::vector<float> Lc(static_cast<size_t>(d) * d), drift(d);
    for (int u = 0; u < d; ++u) {
        for (int k = 0; k < d; ++k) Lc[static_cast<size_t>(u) * d + k] = static_cast<float>(std::sqrt(h) * pf->sigma[u] * L[static_cast<size_t>(u) * d + k]);
        drift[u] = static_cast<float>((pf->mu - 0.5 * pf->sigma[u] * pf->sigma[u]) * h);
    }
    RK_CUDA(cudaMemcpyAsync(d_Lc, Lc.data(), Lc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RK_CUDA(cudaMemcpyAsync(d_drift, drift.data(), d * sizeof(float), cudaMemcpyHostToDevice, s));
    const uint32_t k0 = static_cast<uint32_t>(cf->seed), k1 = static_cast<uint32_t>(cf->seed >> 32);
    const RoundKeys rk = round_keys(k0, k1);
    RK_CUDA(launch_outer(ns, cf->scen_offset, d, d_Lc, d_drift, d_s0, rk, d_Sp, s));

    RiskArgs a{};
    a.d = d;
    a.nopt = no;
    a.s0 = d_s0;
    a.sigma = d_sig;
    a.r = static_cast<float>(pf->r);
    a.dt = static_cast<float>(dt);
    a.horizon_steps = hsteps;
    a.under = d_under;
    a.under_start = d_start;
    a.kind = d_kind;
    a.rem = d_rem;
    a.strike = d_K;
    a.barrier = d_H;
    a.pos = d_pos;
    a.base = d_base;
    a.base_out = d_base;
    a.rk = rk;
    a.scen_off = cf->scen_offset;
    if (cf->method == MC_RISK_NESTED) {
        double *d_contrib;
        RK_CUDA(B.alloc(&d_contrib, ns * d));
        a.inner = cf->base_paths;
        RK_CUDA(launch_nested(a, 1, nullptr, nullptr, s));  // base values at S0, full maturities
        a.inner = cf->inner_paths;
        RK_CUDA(launch_nested(a, ns, d_Sp, d_contrib, s));
        RK_CUDA(launch_sum_under(ns, d, d_contrib, d_pnl, s));
    } else {
        mc_mlp *net = cf->surrogate;
        const MlpLayout &NL = mlp_layout_of(net);
        if (NL.sizes.front() != 5) return fail(MC_EINVAL, "the surrogate must take 5 inputs");
        const int64_t chunk = std::max<int64_t>(1, (int64_t(1) << 20) / no);  // scenarios per evaluation
        float *d_x, *d_y;
        RK_CUDA(B.alloc(&d_x, std::min(ns, chunk) * no * 5));
        RK_CUDA(B.alloc(&d_y, std::min(ns, chunk) * no));
        RK_CUDA(launch_features(a, 1, nullptr, d_x, s));
        int rc = mlp_forward_any(net, d_x, no, d_y, cf->surrogate_precision, s);
        if (rc) return rc;
        RK_CUDA(launch_pnl(a, 1, nullptr, d_y, nullptr, s));  // base values
        for (int64_t s0 = 0; s0 < ns; s0 += chunk) {
            const int64_t nc = std::min(chunk, ns - s0);
            RK_CUDA(launch_features(a, nc, d_Sp + s0 * d, d_x, s));
            rc = mlp_forward_any(net, d_x, nc * no, d_y, cf->surrogate_precision, s);
            if (rc) return rc;
            RK_CUDA(launch_pnl(a, nc, d_Sp + s0 * d, d_y, d_pnl + s0, s));
        }
    }
    RK_CUDA(launch_tail(ns, d_pnl, d_work, np2, cf->alpha, d_res, s));
    double r3[3];
    std::vector<double> base(no);
    RK_CUDA(cudaMemcpyAsync(r3, d_res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    RK_CUDA(cudaMemcpyAsync(base.data(), d_base, no * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (host_pnl) RK_CUDA(cudaMemcpyAsync(host_pnl, d_pnl, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    RK_CUDA(cudaStreamSynchronize(s));
    if (cf->method == MC_RISK_SURROGATE && cf->surrogate_precision == MC_BF16) {
        const int rc = mlp_check_timeout(cf->surrogate, s);
        if (rc) return rc;
    }
    res->var = r3[0];
    res->cvar = r3[1];
    res->n_tail = static_cast<int64_t>(r3[2]);
    double bv = 0.0;
    for (int i = 0; i < no; ++i) bv += h_pos[i] * base[i];
    res->base_value = bv;
    return MC_OK;
}

}  // extern "C"
