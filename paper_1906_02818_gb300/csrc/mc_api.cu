// Host runtime and C ABI (include/mc.h): argument checks, plan set-up (model
// upload, FP64 Cholesky on the device, scaled factor, persistent-grid sizing,
// scratch for per-block partials), kernel dispatch and error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "mc_kernels.cuh"

using namespace gbmc;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define MC_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA, "%s: %s (%s)", \
                        #call, cudaGetErrorName(e_), cudaGetErrorString(e_));                  \
    } while (0)

bool finite_all(const double *p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

int check_model(const mc_model *m)
{
    if (!m) return fail(MC_EINVAL, "model is NULL");
    if (m->kind != MC_GBM && m->kind != MC_HESTON) return fail(MC_EINVAL, "unknown model kind %d", m->kind);
    if (m->d < 1 || m->d > 4096) return fail(MC_EINVAL, "d = %d out of range [1, 4096]", m->d);
    if (!m->s0) return fail(MC_EINVAL, "s0 is NULL");
    if (!std::isfinite(m->r)) return fail(MC_EINVAL, "r is not finite");
    for (int a = 0; a < m->d; ++a)
        if (!(m->s0[a] > 0.0) || !std::isfinite(m->s0[a])) return fail(MC_EINVAL, "s0[%d] must be finite and > 0", a);
    if (m->kind == MC_HESTON) {
        if (m->d != 1) return fail(MC_EINVAL, "Heston requires d == 1");
        if (m->loadings || m->corr) return fail(MC_EINVAL, "Heston takes no correlation or loadings");
        const double v[5] = {m->v0, m->kappa, m->theta, m->xi, m->rho};
        if (!finite_all(v, 5)) return fail(MC_EINVAL, "Heston parameters must be finite");
        if (m->v0 < 0 || m->kappa < 0 || m->theta < 0 || m->xi < 0)
            return fail(MC_EINVAL, "Heston v0, kappa, theta, xi must be >= 0");
        if (!(m->rho > -1.0 && m->rho < 1.0)) return fail(MC_EINVAL, "Heston rho must lie in (-1, 1)");
        return MC_OK;
    }
    if (!m->sigma) return fail(MC_EINVAL, "sigma is NULL");
    for (int a = 0; a < m->d; ++a)
        if (!(m->sigma[a] >= 0.0) || !std::isfinite(m->sigma[a])) return fail(MC_EINVAL, "sigma[%d] must be finite and >= 0", a);
    if (m->weights && !finite_all(m->weights, m->d)) return fail(MC_EINVAL, "weights must be finite");
    if (m->loadings) {
        const int d = m->d, k = m->n_factors;
        if (m->corr) return fail(MC_EINVAL, "give either corr or loadings, not both");
        if (k < 0 || k > kFactorMax) return fail(MC_EUNSUPPORTED, "n_factors = %d outside [0, %d]", k, kFactorMax);
        if (d > kFactorMaxD) return fail(MC_EUNSUPPORTED, "factor model: d = %d exceeds %d", d, kFactorMaxD);
        if (!finite_all(m->loadings, static_cast<int64_t>(d) * k)) return fail(MC_EINVAL, "loadings must be finite");
        for (int i = 0; i < d; ++i) {
            double q = 0.0;
            for (int j = 0; j < k; ++j) q += m->loadings[static_cast<int64_t>(i) * k + j] * m->loadings[static_cast<int64_t>(i) * k + j];
            if (q > 1.0 + 1e-12) return fail(MC_EINVAL, "loadings row %d has norm^2 %g > 1", i, q);
        }
        return MC_OK;
    }
    if (m->corr) {
        const int d = m->d;
        if (!finite_all(m->corr, static_cast<int64_t>(d) * d)) return fail(MC_EINVAL, "corr must be finite");
        for (int i = 0; i < d; ++i) {
            if (std::fabs(m->corr[static_cast<int64_t>(i) * d + i] - 1.0) > 1e-12)
                return fail(MC_EINVAL, "corr[%d][%d] must be 1 (unit diagonal)", i, i);
            for (int j = 0; j < i; ++j) {
                const double a = m->corr[static_cast<int64_t>(i) * d + j], b = m->corr[static_cast<int64_t>(j) * d + i];
                if (std::fabs(a - b) > 1e-12 * (1.0 + std::fabs(a)))
                    return fail(MC_EINVAL, "corr is not symmetric at (%d, %d)", i, j);
                if (std::fabs(a) > 1.0) return fail(MC_EINVAL, "corr[%d][%d] = %g outside [-1, 1]", i, j, a);
            }
        }
    }
    return MC_OK;
}

int check_cfg(const mc_sim_cfg *c, const mc_model *m)
{
    if (!c) return fail(MC_EINVAL, "cfg is NULL");
    if (c->steps < 1) return fail(MC_EINVAL, "steps = %d must be >= 1", c->steps);
    if (!(c->T > 0.0) || !std::isfinite(c->T)) return fail(MC_EINVAL, "T must be finite and > 0");
    if (c->paths < 1) return fail(MC_EINVAL, "paths = %lld must be >= 1", static_cast<long long>(c->paths));
    if (c->path_offset < 0 || c->path_offset + c->paths > (int64_t(1) << 56))
        return fail(MC_EINVAL, "path range must lie in [0, 2^56)");
    if (c->scheme != MC_LOG_EULER && c->scheme != MC_EULER) return fail(MC_EINVAL, "unknown scheme %d", c->scheme);
    if (c->precision < MC_FP32 || c->precision > MC_FP8E4M3) return fail(MC_EINVAL, "unknown precision %d", c->precision);
    if (c->ckpt_every < 0) return fail(MC_EINVAL, "ckpt_every must be >= 0");
    if (m->kind == MC_HESTON && c->precision != MC_FP32)
        return fail(MC_EINVAL, "Heston has no correlation contraction: precision must be MC_FP32");
    if (m->loadings && c->precision != MC_FP32) return fail(MC_EUNSUPPORTED, "factor model: FP32 only");
    if (c->monitoring != MC_DISCRETE && c->monitoring != MC_BRIDGE)
        return fail(MC_EINVAL, "unknown monitoring %d", c->monitoring);
    if (c->monitoring == MC_BRIDGE && (m->kind != MC_GBM || m->d != 1 || c->scheme != MC_LOG_EULER || m->loadings))
        return fail(MC_EUNSUPPORTED, "Brownian-bridge monitoring: single-asset GBM with MC_LOG_EULER only");
    return MC_OK;
}

int build_payoffs(const mc_payoff *p, int np, PayoffSet *ps)
{
    if (np < 0 || np > MC_MAX_PAYOFFS) return fail(MC_EINVAL, "n_payoff = %d out of range [0, %d]", np, MC_MAX_PAYOFFS);
    if (np > 0 && !p) return fail(MC_EINVAL, "payoffs is NULL");
    std::memset(ps, 0, sizeof *ps);
    ps->n = np;
    for (int i = 0; i < np; ++i) {
        const int k = p[i].kind;
        if (k < MC_CALL || k > MC_DI_PUT) return fail(MC_EINVAL, "payoff %d: unknown kind %d", i, k);
        if (!std::isfinite(p[i].strike)) return fail(MC_EINVAL, "payoff %d: strike not finite", i);
        const bool barrier = k >= MC_UO_CALL;
        if (barrier && std::isnan(p[i].barrier)) return fail(MC_EINVAL, "payoff %d: barrier is NaN", i);
        ps->kind[i] = k;
        ps->strike[i] = static_cast<float>(p[i].strike);
        ps->barrier[i] = barrier ? static_cast<float>(p[i].barrier) : INFINITY;
        if (k == MC_ASIAN_CALL || k == MC_ASIAN_PUT) ps->need_avg = 1;
        if (k >= MC_UO_CALL && k <= MC_UI_PUT) ps->need_max = 1;
        if (k >= MC_DO_CALL) ps->need_min = 1;
    }
    return MC_OK;
}

struct DeviceInfo {
    int device = -1;
    int sms = 0;
};

int device_info(DeviceInfo *di)
{
    MC_CUDA(cudaGetDevice(&di->device));
    MC_CUDA(cudaDeviceGetAttribute(&di->sms, cudaDevAttrMultiProcessorCount, di->device));
    return MC_OK;
}

// Persistent single-wave grid: at most `resident` blocks, every thread the
// same number of paths (ppt), grid shrunk so that no block is idle.
void size_grid(int64_t paths, int block, int resident, int *grid, int *ppt)
{
    int64_t g = (paths + block - 1) / block;
    if (resident > 0 && g > resident) g = resident;
    if (g < 1) g = 1;
    int64_t p = (paths + g * block - 1) / (g * block);
    g = (paths + p * block - 1) / (p * block);
    *grid = static_cast<int>(g);
    *ppt = static_cast<int>(p);
}

// Device allocations of the set-up paths come from a cache of freed blocks
// (per device; sizes rounded up to 256 bytes; a request takes the smallest
// free block of at least its size and at most twice it), so that repeated
// calls of the same shape pay neither cudaMalloc nor cudaFree (which also
// synchronises the device).  A block goes back to the cache only when no
// launch can still use it (its owner has synchronised); mc_release_cache()
// hands the cached blocks back to CUDA.
struct CachedBlock {
    void *p;
    size_t size;
    int dev;
};
std::mutex g_cache_mu;
std::vector<CachedBlock> g_free_blocks;
std::unordered_map<void *, CachedBlock> g_live_blocks;

void release_cached(int dev)  // dev < 0: every device; caller holds g_cache_mu
{
    std::vector<CachedBlock> keep;
    for (const CachedBlock &b : g_free_blocks) {
        if (dev < 0 || b.dev == dev) {
            int cur = -1;
            cudaGetDevice(&cur);
            if (cur != b.dev) cudaSetDevice(b.dev);
            cudaFree(b.p);
            if (cur != b.dev) cudaSetDevice(cur);
        } else {
            keep.push_back(b);
        }
    }
    g_free_blocks.swap(keep);
}

cudaError_t dev_alloc_raw(void **p, size_t n)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t sz = n <= 256 ? 256 : (n + 255) & ~static_cast<size_t>(255);
    std::lock_guard<std::mutex> g(g_cache_mu);
    size_t best = static_cast<size_t>(-1), bi = 0;
    for (size_t i = 0; i < g_free_blocks.size(); ++i) {
        const CachedBlock &b = g_free_blocks[i];
        if (b.dev == dev && b.size >= sz && b.size <= 2 * sz && b.size < best) {
            best = b.size;
            bi = i;
        }
    }
    if (best != static_cast<size_t>(-1)) {
        const CachedBlock b = g_free_blocks[bi];
        g_free_blocks[bi] = g_free_blocks.back();
        g_free_blocks.pop_back();
        g_live_blocks[b.p] = b;
        *p = b.p;
        return cudaSuccess;
    }
    e = cudaMalloc(p, sz);
    if (e == cudaErrorMemoryAllocation && !g_free_blocks.empty()) {
        cudaGetLastError();
        release_cached(dev);
        e = cudaMalloc(p, sz);
    }
    if (e != cudaSuccess) return e;
    g_live_blocks[*p] = CachedBlock{*p, sz, dev};
    return cudaSuccess;
}

void dev_free_raw(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_live_blocks.find(p);
    if (it == g_live_blocks.end()) {
        cudaFree(p);
        return;
    }
    g_free_blocks.push_back(it->second);
    g_live_blocks.erase(it);
}

template <class T>
cudaError_t dev_alloc(T **p, size_t n)
{
    return dev_alloc_raw(reinterpret_cast<void **>(p), n);
}

template <class T>
void dfree(T *&p)
{
    dev_free_raw(p);
    p = nullptr;
}

// Waits for every launch of `dev` (the owner of buffers about to return to
// the cache may not have synchronised).
void sync_device(int dev)
{
    if (dev < 0) {
        cudaDeviceSynchronize();
        return;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    if (cur != dev) cudaSetDevice(cur);
}

// One device allocation carved into 256-byte aligned pieces, freed on scope exit.
struct DeviceArena {
    unsigned char *base = nullptr;
    size_t used = 0;
    bool idle = false;  // set once the owner's stream has been synchronised
    ~DeviceArena()
    {
        if (!base) return;
        if (!idle) {
            int dev = -1;
            cudaGetDevice(&dev);
            sync_device(dev);
        }
        dev_free_raw(base);
    }
    static size_t up(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }
    template <class T>
    T *take(size_t count)
    {
        T *p = reinterpret_cast<T *>(base + used);
        used += up(count * sizeof(T));
        return p;
    }
};


}  // namespace

// Polls of a bounded mbarrier wait before a kernel gives up (GBMC_WAIT_CAP
// overrides; each poll suspends for at most a few microseconds).
int gbmc::check_price_args(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *p, int np, PayoffSet *ps)
{
    int rc;
    if ((rc = check_model(m)) || (rc = check_cfg(c, m)) || (rc = build_payoffs(p, np, ps))) return rc;
    return MC_OK;
}

// GBMC_TEST_STALL=1 sets the cap's top bit: each tensor-core kernel then
// starts with a wait that nothing completes and fails by design (the test of
// the failure path; no asynchronous work is in flight at that point).
uint32_t gbmc::mbar_wait_cap()
{
    uint32_t cap = 1u << 22;
    const char *e = std::getenv("GBMC_WAIT_CAP");
    if (e && *e) {
        const long v = std::strtol(e, nullptr, 10);
        if (v > 0) cap = static_cast<uint32_t>(v < 0x7fffffffL ? v : 0x7fffffffL);
    }
    const char *st = std::getenv("GBMC_TEST_STALL");
    if (st && st[0] == '1') cap |= 0x80000000u;
    return cap;
}

namespace {
std::vector<gbmc::DebugReader> &debug_readers()
{
    static std::vector<gbmc::DebugReader> v;  // filled while the library loads
    return v;
}
}  // namespace

void gbmc::debug_register(DebugReader fn) { debug_readers().push_back(fn); }

int gbmc::set_last_error(int code, const char *msg)
{
    g_err = msg ? msg : "";
    return code;
}

enum KernelKind { K_GBM1D = 0, K_BASKET_FP32 = 1, K_HESTON = 2, K_BASKET_TC = 3, K_BASKET_BIG = 4, K_FACTOR = 5 };

struct mc_plan {
    int device = -1;
    KernelKind kk = K_GBM1D;
    int np = 0;
    int grid = 0, block = 256;
    int D = 0;
    Gbm1dArgs g1{};
    BasketArgs bk{};
    HestonArgs hs{};
    TcArgs tc{};
    TcConst tcc{};
    BigArgs bg{};
    FactorArgs fa{};
    float *dcol = nullptr;  // large baskets and factor models: per-column float arrays
    int prec = MC_FP32;
    uint8_t *bimg = nullptr;
    unsigned int *err = nullptr;
    std::vector<unsigned char> cst;
    float *partials = nullptr;
    unsigned int *ticket = nullptr;
    mc_result *dout = nullptr;
    double *dcorr = nullptr, *dL = nullptr, *dsig = nullptr;
    float *dLp = nullptr, *ddrift = nullptr;
    int *dstatus = nullptr;
    float *ckpt = nullptr;
    double *dsums = nullptr;

    bool idle = false;  // set once every launch that uses the buffers has completed

    ~mc_plan()
    {
        if (!idle) sync_device(device);
        dfree(partials); dfree(ticket); dfree(dout); dfree(dcorr); dfree(dL); dfree(dsig);
        dfree(dLp); dfree(ddrift); dfree(dstatus); dfree(bimg); dfree(err); dfree(ckpt); dfree(dcol);
        dfree(dsums);
    }
};

namespace {

// Large-basket set-up (64 < d <= 512, or any basket when Greeks are asked
// for): FP64 Cholesky on the device, then the tensor-core factor chunks and
// epilogue constants, or the packed FP32 factor; per-column arrays; grid.
int big_setup(mc_plan *P, const mc_model *m, const mc_sim_cfg *c, const PayoffSet &ps, const PathRun &run,
              bool greeks, cudaStream_t s)
{
    const int d = m->d;
    if (d > kBigMaxD) return fail(MC_EUNSUPPORTED, "d = %d beyond %d", d, kBigMaxD);
    if (c->scheme != MC_LOG_EULER) return fail(MC_EUNSUPPORTED, "baskets with d > 64 use the log-Euler scheme");
    for (int i = 0; i < ps.n; ++i)
        if (ps.kind[i] != MC_CALL && ps.kind[i] != MC_PUT)
            return fail(MC_EUNSUPPORTED, "baskets with d > 64 (and basket Greeks) take European calls and puts");
    const bool tcp = c->precision != MC_FP32;
    P->kk = K_BASKET_BIG;
    P->prec = c->precision;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const size_t dd = static_cast<size_t>(d) * d;
    MC_CUDA(dev_alloc(&P->dcorr, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P->dL, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P->dsig, d * sizeof(double)));
    MC_CUDA(dev_alloc(&P->dstatus, sizeof(int)));
    MC_CUDA(dev_alloc(&P->err, sizeof(unsigned int)));
    MC_CUDA(cudaMemsetAsync(P->err, 0, sizeof(unsigned int), s));
    // per-column floats: cs, mdrift, vscale, drift, ws0, w, s0, sigma (8 x d)
    MC_CUDA(dev_alloc(&P->dcol, 8 * static_cast<size_t>(kBigMaxD) * sizeof(float)));
    float *col = P->dcol;
    std::vector<double> corr(dd, 0.0);
    if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
    else for (int k = 0; k < d; ++k) corr[static_cast<size_t>(k) * d + k] = 1.0;
    MC_CUDA(cudaMemcpyAsync(P->dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(P->dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_cholesky(d, P->dcorr, P->dL, P->dstatus, s));
    if (tcp) {
        MC_CUDA(dev_alloc(&P->bimg, big_bimg_bytes(P->prec)));
        MC_CUDA(cudaMemsetAsync(P->bimg, 0, big_bimg_bytes(P->prec), s));
        MC_CUDA(launch_big_prep(P->prec, d, P->dL, P->dsig, M_LOG2E, sdt, m->r, dt, c->steps, P->bimg, col,
                                col + kBigMaxD, col + 2 * kBigMaxD, s));
    } else {
        const size_t D = static_cast<size_t>(wide_width(d));
        MC_CUDA(dev_alloc(&P->dLp, D * D * sizeof(float)));
        MC_CUDA(launch_wide_prep(d, P->dL, P->dsig, sdt, m->r, dt, P->dLp, col + 3 * kBigMaxD, s));
    }
    std::vector<float> h(4 * static_cast<size_t>(kBigMaxD), 0.0f);
    for (int k = 0; k < d; ++k) {
        const double w = m->weights ? m->weights[k] : 1.0 / d;
        h[k] = static_cast<float>(w * m->s0[k]);
        h[kBigMaxD + k] = static_cast<float>(w);
        h[2 * kBigMaxD + k] = static_cast<float>(m->s0[k]);
        h[3 * kBigMaxD + k] = static_cast<float>(m->sigma[k]);
    }
    MC_CUDA(cudaMemcpyAsync(col + 4 * kBigMaxD, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    int status = 0;
    MC_CUDA(cudaMemcpyAsync(&status, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    BigArgs &b = P->bg;
    b.run = run;
    b.d = d;
    b.exact4 = d % 4 == 0;
    b.greeks = greeks ? 1 : 0;
    b.bimg = P->bimg;
    b.Lp = P->dLp;
    b.cs = col;
    b.mdrift = col + kBigMaxD;
    b.vscale = col + 2 * kBigMaxD;
    b.drift = col + 3 * kBigMaxD;
    b.ws0 = col + 4 * kBigMaxD;
    b.w = col + 5 * kBigMaxD;
    b.s0 = col + 6 * kBigMaxD;
    b.sigma = col + 7 * kBigMaxD;
    b.T = static_cast<float>(c->T);
    b.sdt = static_cast<float>(sdt);
    b.pay = ps;
    b.err = P->err;
    b.disc = std::exp(-m->r * c->T);
    b.wait_cap = mbar_wait_cap();
    P->grid = basket_big_grid(P->prec, c->paths);
    if (P->grid <= 0) return fail(MC_ECUDA, "large-basket kernel cannot be resident");
    const int nvals = ps.n + (greeks ? 2 * d + 1 : 0);
    P->np = nvals;
    MC_CUDA(dev_alloc(&P->partials, static_cast<size_t>(P->grid) * nvals * 2 * sizeof(float)));
    MC_CUDA(dev_alloc(&P->ticket, sizeof(unsigned int)));
    MC_CUDA(cudaMemsetAsync(P->ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(dev_alloc(&P->dout, static_cast<size_t>(nvals) * sizeof(mc_result)));
    b.partials = P->partials;
    b.ticket = P->ticket;
    b.out = P->dout;
    return MC_OK;
}

// Factor-model basket: B', e', drift and the basket columns in FP64 on the
// host, padded to 256 G assets, then one upload.
int factor_setup(mc_plan *P, const mc_model *m, const mc_sim_cfg *c, const PayoffSet &ps, const PathRun &run,
                 const ReduceArgs &red, const DeviceInfo &di, cudaStream_t s)
{
    const int d = m->d, k = m->n_factors, G = (d + 255) / 256, dp = 256 * G;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const double cfac = c->scheme == MC_LOG_EULER ? M_LOG2E : 1.0;
    std::vector<float> h(static_cast<size_t>(k + 7) * dp, 0.0f);
    float *Bp = h.data(), *ep = Bp + static_cast<size_t>(k) * dp, *dr = ep + dp, *ws0 = dr + dp, *w = ws0 + dp,
          *s0 = w + dp, *sgm = s0 + dp;
    for (int a = 0; a < dp; ++a) s0[a] = sgm[a] = 1.0f;  // padded assets: inert
    for (int a = 0; a < d; ++a) {
        const double sg = m->sigma[a], cs = cfac * sdt * sg;
        double q = 0.0;
        for (int j = 0; j < k; ++j) {
            const double b = m->loadings[static_cast<int64_t>(a) * k + j];
            q += b * b;
            Bp[static_cast<size_t>(j) * dp + a] = static_cast<float>(cs * b);
        }
        ep[a] = static_cast<float>(cs * std::sqrt(std::max(0.0, 1.0 - q)));
        dr[a] = static_cast<float>(c->scheme == MC_LOG_EULER ? cfac * (m->r - 0.5 * sg * sg) * dt : m->r * dt);
        const double wa = m->weights ? m->weights[a] : 1.0 / d;
        ws0[a] = static_cast<float>(wa * m->s0[a]);
        w[a] = static_cast<float>(wa);
        s0[a] = static_cast<float>(m->s0[a]);
        sgm[a] = static_cast<float>(sg);
    }
    MC_CUDA(dev_alloc(&P->dcol, h.size() * sizeof(float)));
    MC_CUDA(cudaMemcpyAsync(P->dcol, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    P->kk = K_FACTOR;
    FactorArgs &f = P->fa;
    f.run = run;
    f.d = d;
    f.k = k;
    f.G = G;
    f.scheme = c->scheme;
    f.exact4 = (k % 4 == 0 && d % 4 == 0) ? 1 : 0;
    f.Bp = P->dcol;
    f.ep = P->dcol + static_cast<size_t>(k) * dp;
    f.drift = f.ep + dp;
    f.ws0 = f.drift + dp;
    f.w = f.ws0 + dp;
    f.s0 = f.w + dp;
    f.sigma = f.s0 + dp;
    f.greeks = 0;
    f.T = static_cast<float>(c->T);
    f.r = static_cast<float>(m->r);
    f.gpart = nullptr;
    f.pay = ps;
    f.red = red;
    const int occ = factor_occupancy(f);
    if (occ <= 0) return fail(MC_ECUDA, "factor-model kernel cannot be resident");
    const int per = factor_paths_per_cta(f);
    const int64_t tiles = (c->paths + per - 1) / per;
    P->grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(occ) * di.sms));
    P->block = 256;
    const int np = ps.n;
    MC_CUDA(dev_alloc(&P->partials, static_cast<size_t>(P->grid) * np * 2 * sizeof(float)));
    MC_CUDA(dev_alloc(&P->ticket, sizeof(unsigned int)));
    MC_CUDA(cudaMemsetAsync(P->ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(dev_alloc(&P->dout, static_cast<size_t>(np) * sizeof(mc_result)));
    f.red.partials = P->partials;
    f.red.ticket = P->ticket;
    f.red.out = P->dout;
    return MC_OK;
}

// Shared set-up of mc_plan_create and mc_simulate.  save != nullptr selects
// the materialising kernels (no payoffs, no reduction).
int plan_setup(mc_plan *P, const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pays, int np,
               float *save, int save_every, cudaStream_t s)
{
    int rc;
    if ((rc = check_model(m)) || (rc = check_cfg(c, m))) return rc;
    PayoffSet ps;
    if ((rc = build_payoffs(pays, np, &ps))) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    P->device = di.device;
    P->np = np;

    PathRun run{};
    run.paths = c->paths;
    run.path_offset = c->path_offset;
    set_seed(run, c->seed);
    run.steps = c->steps;
    run.save = save;
    run.save_every = save_every > 0 ? save_every : 1;

    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const double disc = std::exp(-m->r * c->T);
    ReduceArgs red{};
    red.paths = c->paths;
    red.disc = disc;
    int resident = 0;

    if (m->kind == MC_HESTON) {
        P->kk = K_HESTON;
        HestonArgs &h = P->hs;
        h.run = run;
        h.s0 = static_cast<float>(m->s0[0]);
        h.v0 = static_cast<float>(m->v0);
        h.r = static_cast<float>(m->r);
        h.kappa = static_cast<float>(m->kappa);
        h.theta = static_cast<float>(m->theta);
        h.xi = static_cast<float>(m->xi);
        h.rho = static_cast<float>(m->rho);
        h.rhoc = static_cast<float>(std::sqrt(1.0 - m->rho * m->rho));
        h.dt = static_cast<float>(dt);
        h.pay = ps;
        h.red = red;
        resident = heston_occupancy(h, P->block) * di.sms;
    } else if (m->loadings) {
        if (save) return fail(MC_EUNSUPPORTED, "factor model: paths are not materialised");
        if (np < 1) return fail(MC_EINVAL, "n_payoff must be >= 1");
        return factor_setup(P, m, c, ps, run, red, di, s);
    } else if (m->d == 1) {
        P->kk = K_GBM1D;
        if (m->corr && std::fabs(m->corr[0] - 1.0) > 1e-12) return fail(MC_EINVAL, "corr[0] must be 1");
        Gbm1dArgs &g = P->g1;
        g.run = run;
        g.scheme = c->scheme;
        const double sg = m->sigma[0];
        const double w = m->weights ? m->weights[0] : 1.0;
        // U = w S for a one-asset basket; the kernel simulates S and the
        // weight is folded into S0 (U is linear in S0 under both schemes).
        g.s0 = static_cast<float>(save ? m->s0[0] : w * m->s0[0]);
        if (c->scheme == MC_LOG_EULER) {
            g.a = static_cast<float>(M_LOG2E * (m->r - 0.5 * sg * sg) * dt);
            g.b = static_cast<float>(M_LOG2E * sg * sdt);
            // bridge in log2 units: (log2 e)^2 sigma^2 dt (-2 ln U) = -cb lg2 U
            g.bridge = c->monitoring == MC_BRIDGE && !save && ps.n > 0 ? 1 : 0;
            g.cb = static_cast<float>(2.0 * M_LOG2E * sg * sg * dt);
        } else {
            g.a = static_cast<float>(m->r * dt);
            g.b = static_cast<float>(sg * sdt);
        }
        g.pay = ps;
        g.red = red;
        resident = gbm1d_occupancy(g, P->block) * di.sms;
    } else if (m->d > 64) {
        if (save) return fail(MC_EUNSUPPORTED, "paths are materialised for d <= 64");
        return big_setup(P, m, c, ps, run, false, s);
    } else {
        const int d = m->d;
        const bool tcpath = c->precision != MC_FP32;
        if (tcpath && save)
            return fail(MC_EUNSUPPORTED, "paths are materialised by the FP32 contraction only");
        const int D = tcpath ? 64 : basket_fp32_width(d);
        if (!D) return fail(MC_EUNSUPPORTED, "FP32 contraction supports d <= 64 (got %d)", d);
        P->D = D;
        const size_t dd = static_cast<size_t>(d) * d;
        const size_t tri = static_cast<size_t>(d) * (d + 1) / 2;
        MC_CUDA(dev_alloc(&P->dcorr, dd * sizeof(double)));
        MC_CUDA(dev_alloc(&P->dL, dd * sizeof(double)));
        MC_CUDA(dev_alloc(&P->dsig, d * sizeof(double)));
        MC_CUDA(dev_alloc(&P->dLp, (tcpath ? 64 : tri) * sizeof(float)));
        MC_CUDA(dev_alloc(&P->ddrift, (tcpath ? 64 : d) * sizeof(float)));
        MC_CUDA(dev_alloc(&P->dstatus, sizeof(int)));
        std::vector<double> corr(dd, 0.0);
        if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
        else for (int a = 0; a < d; ++a) corr[static_cast<size_t>(a) * d + a] = 1.0;
        MC_CUDA(cudaMemcpyAsync(P->dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
        MC_CUDA(cudaMemcpyAsync(P->dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
        MC_CUDA(launch_cholesky(d, P->dcorr, P->dL, P->dstatus, s));
        const double cfac = c->scheme == MC_LOG_EULER ? M_LOG2E : 1.0;
        int status = 0;
        if (tcpath) {
            // Quantised, swizzled factor tile + per-column scales (FP64 -> operand type).
            P->kk = K_BASKET_TC;
            P->prec = c->precision;
            MC_CUDA(dev_alloc(&P->bimg, tc_bimg_bytes(P->prec)));
            MC_CUDA(dev_alloc(&P->err, sizeof(unsigned int)));
            MC_CUDA(cudaMemsetAsync(P->err, 0, sizeof(unsigned int), s));
            MC_CUDA(launch_tc_prep(P->prec, d, P->dL, P->dsig, cfac, sdt, m->r, dt, c->scheme, P->bimg, P->dLp,
                                   P->ddrift, s));
            std::vector<float> cs(64), drift(64);
            MC_CUDA(cudaMemcpyAsync(&status, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(cs.data(), P->dLp, 64 * sizeof(float), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(drift.data(), P->ddrift, 64 * sizeof(float), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
            TcConst &k = P->tcc;
            std::memset(&k, 0, sizeof k);
            for (int a = 0; a < 64; ++a) {
                k.cs[a] = cs[a];
                k.drift[a] = drift[a];
                if (a < d) {
                    const double w = m->weights ? m->weights[a] : 1.0 / d;
                    k.ws0[a] = static_cast<float>(w * m->s0[a]);
                    k.w[a] = static_cast<float>(w);
                    k.s0[a] = static_cast<float>(m->s0[a]);
                } else {
                    k.s0[a] = 1.0f;  // padded columns: zero weight, inert state
                }
            }
            TcArgs &ta = P->tc;
            ta.run = run;
            ta.d = d;
            ta.scheme = c->scheme;
            ta.bimg = P->bimg;
            ta.pay = ps;
            ta.red = red;
            ta.red.err = P->err;
            ta.err = P->err;
            const uint32_t cap = mbar_wait_cap();
            ta.wait_cap = cap & 0x7fffffffu;
            ta.stall = cap >> 31;
            P->block = 128;
            resident = basket_tc_occupancy(P->prec, ta) * di.sms;
        } else {
            P->kk = K_BASKET_FP32;
            // Large runs: one block per SM, as many rounds of paths as 640
            // threads need, the block trimmed (to whole warps) so that those
            // rounds cover the paths on every SM; small runs (or a trimmed
            // block under 16 warps): blocks of 128, 5 per SM, to spread them.
            const int64_t per_round = static_cast<int64_t>(640) * di.sms;
            const int64_t rounds = (c->paths + per_round - 1) / per_round;
            const int64_t per_sm = (c->paths + rounds * di.sms - 1) / (rounds * di.sms);
            const int trimmed = static_cast<int>(std::min<int64_t>(640, (per_sm + 31) / 32 * 32));
            P->block = (c->paths >= 2 * per_round || trimmed >= 512) && c->paths >= per_round ? trimmed : 128;
            MC_CUDA(launch_scale_factor(d, P->dL, P->dsig, cfac, sdt, m->r, dt, c->scheme, P->dLp, P->ddrift, s));
            std::vector<float> Lp(tri), drift(d);
            MC_CUDA(cudaMemcpyAsync(&status, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(Lp.data(), P->dLp, tri * sizeof(float), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaMemcpyAsync(drift.data(), P->ddrift, d * sizeof(float), cudaMemcpyDeviceToHost, s));
            MC_CUDA(cudaStreamSynchronize(s));
            if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
            // Pack the launch-parameter block: rows of width D, zero beyond d.
            P->cst.assign(basket_const_bytes(D), 0);
            size_t oL, oDr, oWs, oW, oS;
            basket_const_offsets(D, &oL, &oDr, &oWs, &oW, &oS);
            float *cL = reinterpret_cast<float *>(P->cst.data() + oL);  // column pairs, see BasketConst
            float *cDr = reinterpret_cast<float *>(P->cst.data() + oDr);
            float *cWs = reinterpret_cast<float *>(P->cst.data() + oWs);
            float *cW = reinterpret_cast<float *>(P->cst.data() + oW);
            float *cS = reinterpret_cast<float *>(P->cst.data() + oS);
            for (int k = 0; k < d; ++k)
                for (int q = k / 2; q < D / 2; ++q)
                    for (int h = 0; h < 2; ++h) {
                        const int a = 2 * q + h;  // row; zero above the diagonal and beyond d
                        if (a >= k && a < d)
                            cL[2 * (basket_pair_base(D, k) + q - k / 2) + h] = Lp[static_cast<size_t>(a) * (a + 1) / 2 + k];
                    }
            for (int a = 0; a < d; ++a) {
                const double w = m->weights ? m->weights[a] : 1.0 / d;
                cDr[a] = drift[a];
                cWs[a] = static_cast<float>(w * m->s0[a]);
                cW[a] = static_cast<float>(w);
                cS[a] = static_cast<float>(m->s0[a]);
            }
            BasketArgs &b = P->bk;
            b.run = run;
            b.d = d;
            b.scheme = c->scheme;
            b.pay = ps;
            b.red = red;
            resident = basket_fp32_occupancy(D, b, P->block) * di.sms;
        }
    }
    if (resident <= 0) return fail(MC_ECUDA, "kernel cannot be resident (occupancy query failed)");
    int ppt = 1;
    if (P->kk == K_BASKET_TC) {
        const int64_t tiles = (c->paths + 127) / 128;
        P->grid = static_cast<int>(tiles < resident ? tiles : resident);
    } else {
        size_grid(c->paths, P->block, resident, &P->grid, &ppt);
    }
    P->g1.run.ppt = ppt;
    P->bk.run.ppt = ppt;
    P->hs.run.ppt = ppt;
    if (np > 0) {
        MC_CUDA(dev_alloc(&P->partials, static_cast<size_t>(P->grid) * np * 2 * sizeof(float)));
        MC_CUDA(dev_alloc(&P->ticket, sizeof(unsigned int)));
        MC_CUDA(cudaMemsetAsync(P->ticket, 0, sizeof(unsigned int), s));
        MC_CUDA(dev_alloc(&P->dout, static_cast<size_t>(np) * sizeof(mc_result)));
        for (ReduceArgs *r : {&P->g1.red, &P->bk.red, &P->hs.red, &P->tc.red}) {
            r->partials = P->partials;
            r->ticket = P->ticket;
            r->out = P->dout;
        }
    }
    return MC_OK;
}

int plan_launch(mc_plan *P, mc_result *dev_out, cudaStream_t s)
{
    P->idle = false;
    for (ReduceArgs *r : {&P->g1.red, &P->bk.red, &P->hs.red, &P->tc.red}) r->out = dev_out ? dev_out : P->dout;
    switch (P->kk) {
    case K_GBM1D: MC_CUDA(launch_gbm1d(P->g1, P->grid, P->block, s)); break;
    case K_BASKET_FP32: MC_CUDA(launch_basket_fp32(P->D, P->bk, P->cst.data(), P->grid, P->block, s)); break;
    case K_HESTON: MC_CUDA(launch_heston(P->hs, P->grid, P->block, s)); break;
    case K_BASKET_TC: MC_CUDA(launch_basket_tc(P->prec, P->tc, P->tcc, P->grid, s)); break;
    case K_BASKET_BIG:
        P->bg.out = dev_out ? dev_out : P->dout;
        MC_CUDA(launch_basket_big(P->prec, P->bg, P->grid, s));
        break;
    case K_FACTOR:
        P->fa.red.out = dev_out ? dev_out : P->dout;
        MC_CUDA(launch_factor(P->fa, P->grid, s));
        break;
    }
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_version(void) { return MC_VERSION; }

int mc_release_cache(void)
{
    std::lock_guard<std::mutex> g(g_cache_mu);
    release_cached(-1);
    return MC_OK;
}

const char *mc_last_error(void) { return g_err.c_str(); }

int mc_plan_create(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs, int32_t n_payoff,
                   mc_plan **plan, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: plan set-up");
    if (!plan) return fail(MC_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (n_payoff < 1) return fail(MC_EINVAL, "n_payoff must be >= 1");
    mc_plan *P = new (std::nothrow) mc_plan();
    if (!P) return fail(MC_ENOMEM, "host allocation failed");
    int rc = plan_setup(P, model, cfg, payoffs, n_payoff, nullptr, 0, static_cast<cudaStream_t>(stream));
    if (rc) {
        delete P;
        return rc;
    }
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        delete P;
        return fail(MC_ECUDA, "set-up: %s", cudaGetErrorString(e));
    }
    *plan = P;
    return MC_OK;
}

int mc_plan_execute(mc_plan *plan, mc_result *dev_out, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: plan execute");
    if (!plan) return fail(MC_EINVAL, "plan is NULL");
    if (!dev_out) return fail(MC_EINVAL, "dev_out is NULL");
    int dev = -1;
    MC_CUDA(cudaGetDevice(&dev));
    if (dev != plan->device) return fail(MC_EINVAL, "plan belongs to device %d, current is %d", plan->device, dev);
    return plan_launch(plan, dev_out, static_cast<cudaStream_t>(stream));
}

int mc_plan_destroy(mc_plan *plan)
{
    delete plan;
    return MC_OK;
}

int mc_plan_launches(const mc_plan *plan) { return plan ? 1 : 0; }

int mc_debug_status(uint32_t *violations, uint32_t *first_site, int64_t *first_index)
{
#ifdef GBMC_DEBUG
    if (!violations || !first_site || !first_index) return fail(MC_EINVAL, "outputs must be set");
    MC_CUDA(cudaDeviceSynchronize());
    uint32_t total = 0;
    unsigned long long first = 0;
    for (DebugReader fn : debug_readers()) {
        unsigned long long f = 0;
        unsigned c = 0;
        if (fn(&f, &c) != 0) return fail(MC_ECUDA, "reading a debug word failed");
        total += c;
        if (!first && f) first = f;
    }
    *violations = total;
    *first_site = static_cast<uint32_t>(first >> 48);
    *first_index = static_cast<int64_t>(first & 0xFFFFFFFFFFFFull);
    return MC_OK;
#else
    (void)violations; (void)first_site; (void)first_index;
    return fail(MC_EUNSUPPORTED, "this is a release build without bounds checks (build with GBMC_DEBUG)");
#endif
}

// Eq. 3 over a union of disjoint path ranges.  A run over N paths reported
// price = e^{-rT} S1 / N and se = e^{-rT} sqrt((S2 / N - (S1 / N)^2) / (N - 1))
// (S1, S2 the sums of f and f^2), so (N mean, N mean(f^2), N) in discounted
// units are recovered exactly up to rounding, add over runs, and give back
// the estimator and its standard error of the union.
int mc_moments(const mc_result *res, int32_t n_payoff, int64_t paths, double *moments)
{
    if (!res || !moments || n_payoff < 1 || paths < 1) return fail(MC_EINVAL, "res, moments set; n_payoff, paths >= 1");
    const double n = static_cast<double>(paths);
    for (int i = 0; i < n_payoff; ++i) {
        const double m = res[i].price, se = res[i].se;
        if (!std::isfinite(m) || !std::isfinite(se) || se < 0.0) return fail(MC_EINVAL, "result %d is not finite", i);
        const double m2 = paths > 1 ? se * se * (n - 1.0) + m * m : m * m;
        moments[3 * i] = n * m;
        moments[3 * i + 1] = n * m2;
        moments[3 * i + 2] = n;
    }
    return MC_OK;
}

int mc_combine(const double *moments, int32_t n_payoff, mc_result *out)
{
    if (!moments || !out || n_payoff < 1) return fail(MC_EINVAL, "moments, out set; n_payoff >= 1");
    for (int i = 0; i < n_payoff; ++i)
        if (!(moments[3 * i + 2] >= 1.0) || !std::isfinite(moments[3 * i]) || !std::isfinite(moments[3 * i + 1]))
            return fail(MC_EINVAL, "moments of payoff %d: path count < 1 or sums not finite", i);
    for (int i = 0; i < n_payoff; ++i) {
        const double n = moments[3 * i + 2], m = moments[3 * i] / n;
        const double var = std::fmax(moments[3 * i + 1] / n - m * m, 0.0);
        out[i].price = m;
        out[i].se = n > 1.0 ? std::sqrt(var / (n - 1.0)) : 0.0;
    }
    return MC_OK;
}

int mc_price(const mc_model *model, const mc_sim_cfg *cfg, const mc_payoff *payoffs, int32_t n_payoff,
             mc_result *out, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_price");
    if (!out) return fail(MC_EINVAL, "out is NULL");
    mc_plan *P = nullptr;
    int rc = mc_plan_create(model, cfg, payoffs, n_payoff, &P, stream);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = plan_launch(P, P->dout, s);
    std::vector<mc_result> tmp(n_payoff);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(tmp.data(), P->dout, n_payoff * sizeof(mc_result), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(MC_ECUDA, "mc_price: %s", cudaGetErrorString(e));
        else P->idle = true;
    }
    if (!rc && P->err) {
        unsigned int e = 0;
        if (cudaMemcpy(&e, P->err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = fail(MC_ECUDA, "mc_price: reading the wait status failed");
        else if (e)
            rc = fail(MC_ETIMEOUT, "a bounded wait on the tensor-core pipeline gave up");
    }
    if (!rc) std::memcpy(out, tmp.data(), n_payoff * sizeof(mc_result));
    delete P;
    return rc;
}

int32_t mc_greek_count(const mc_model *model)
{
    if (!model) return fail(MC_EINVAL, "model is NULL");
    return model->kind == MC_HESTON ? 7 : 2 * model->d + 1;
}

int mc_greeks(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pays, int32_t np, mc_result *prices,
              mc_result *greeks, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_greeks");
    int rc;
    if (!greeks) return fail(MC_EINVAL, "greeks is NULL");
    if ((rc = check_model(m)) || (rc = check_cfg(c, m))) return rc;
    if (np < 1) return fail(MC_EINVAL, "n_payoff must be >= 1");
    PayoffSet ps;
    if ((rc = build_payoffs(pays, np, &ps))) return rc;
    if (m->loadings) {
        // factor model: delta_n, vega_n, rho of a European basket call or put
        if (c->scheme != MC_LOG_EULER) return fail(MC_EUNSUPPORTED, "factor-model Greeks use the log-Euler scheme");
        if (np != 1 || (ps.kind[0] != MC_CALL && ps.kind[0] != MC_PUT))
            return fail(MC_EUNSUPPORTED, "factor-model Greeks take exactly one European call or put");
        for (int k = 0; k < m->d; ++k)
            if (!(m->sigma[k] > 0.0)) return fail(MC_EINVAL, "factor-model Greeks need sigma > 0 for every asset");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        mc_plan P;
        if ((rc = plan_setup(&P, m, c, pays, np, nullptr, 1, s))) return rc;
        FactorArgs &f = P.fa;
        f.greeks = 1;
        const int occ = factor_occupancy(f);
        if (occ <= 0) return fail(MC_ECUDA, "factor-model Greeks kernel cannot be resident");
        const int per = factor_paths_per_cta(f);
        DeviceInfo di;
        if ((rc = device_info(&di))) return rc;
        // at most the plan's grid (its reduction buffers are sized for it)
        const int64_t tiles = (c->paths + per - 1) / per;
        P.grid = static_cast<int>(std::min(std::min(tiles, static_cast<int64_t>(occ) * di.sms),
                                           static_cast<int64_t>(P.grid)));
        const int G = 2 * m->d + 1;
        DeviceArena ar;
        MC_CUDA(dev_alloc(&ar.base, DeviceArena::up(static_cast<size_t>(P.grid) * G * 2 * sizeof(float)) +
                                        DeviceArena::up(G * sizeof(mc_result))));
        f.gpart = ar.take<float>(static_cast<size_t>(P.grid) * G * 2);
        mc_result *dg = ar.take<mc_result>(G);
        if ((rc = plan_launch(&P, P.dout, s))) return rc;
        MC_CUDA(launch_factor_greeks_finish(f, P.grid, std::exp(-m->r * c->T), dg, s));
        std::vector<mc_result> hg(G);
        mc_result pr;
        MC_CUDA(cudaMemcpyAsync(&pr, P.dout, sizeof pr, cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaMemcpyAsync(hg.data(), dg, G * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        P.idle = true;
        ar.idle = true;
        if (prices) prices[0] = pr;
        for (int k = 0; k < G; ++k) greeks[k] = hg[k];
        return MC_OK;
    }
    for (int i = 0; i < np; ++i)
        if (ps.kind[i] > MC_ASIAN_PUT)
            return fail(MC_EUNSUPPORTED, "payoff %d: barrier payoffs have no pathwise Greek", i);
    if (m->kind == MC_GBM && m->d > 1) {
        // basket: delta_n, vega_n, rho of a European call or put
        if (np != 1) return fail(MC_EINVAL, "basket Greeks take exactly one payoff");
        for (int k = 0; k < m->d; ++k)
            if (!(m->sigma[k] > 0.0)) return fail(MC_EINVAL, "basket Greeks need sigma > 0 for every asset");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        PathRun run{};
        run.paths = c->paths;
        run.path_offset = c->path_offset;
        set_seed(run, c->seed);
        run.steps = c->steps;
        run.save_every = 1;
        mc_plan P;
        if ((rc = big_setup(&P, m, c, ps, run, true, s))) return rc;
        if ((rc = plan_launch(&P, P.dout, s))) return rc;
        const int G = 2 * m->d + 1;
        std::vector<mc_result> tmp(1 + G);
        MC_CUDA(cudaMemcpyAsync(tmp.data(), P.dout, tmp.size() * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        P.idle = true;
        unsigned int e = 0;
        MC_CUDA(cudaMemcpy(&e, P.err, sizeof e, cudaMemcpyDeviceToHost));
        if (e) return fail(MC_ETIMEOUT, "a bounded wait on the tensor-core pipeline gave up");
        if (prices) prices[0] = tmp[0];
        for (int k = 0; k < G; ++k) greeks[k] = tmp[1 + k];
        return MC_OK;
    }
    if (m->kind == MC_GBM && c->scheme != MC_LOG_EULER)
        return fail(MC_EUNSUPPORTED, "GBM Greeks are computed for the log-Euler scheme");
    const int K = c->ckpt_every ? c->ckpt_every : 32;
    if (m->kind == MC_HESTON && (K < 1 || K > 64)) return fail(MC_EINVAL, "ckpt_every = %d outside [1, 64]", K);
    const int G = mc_greek_count(m);
    const int nv = np * (G + 1);
    if (nv * 2 * 4 * static_cast<int>(sizeof(AccSlot)) > 48 * 1024) return fail(MC_EINVAL, "too many payoffs for one Greeks launch");
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const double w = m->weights ? m->weights[0] : 1.0;
    GreeksArgs a{};
    a.run.paths = c->paths;
    a.run.path_offset = c->path_offset;
    set_seed(a.run, c->seed);
    a.run.steps = c->steps;
    a.run.save_every = 1;
    a.model = m->kind;
    a.s0 = static_cast<float>(m->s0[0]);
    a.s0w = static_cast<float>(w * m->s0[0]);
    a.r = static_cast<float>(m->r);
    a.dt = static_cast<float>(dt);
    a.sdt = static_cast<float>(sdt);
    a.T = static_cast<float>(c->T);
    if (m->kind == MC_GBM) {
        const double sg = m->sigma[0];
        a.sigma = static_cast<float>(sg);
        a.a2 = static_cast<float>(M_LOG2E * (m->r - 0.5 * sg * sg) * dt);
        a.b2 = static_cast<float>(M_LOG2E * sg * sdt);
    } else {
        a.v0 = static_cast<float>(m->v0);
        a.kappa = static_cast<float>(m->kappa);
        a.theta = static_cast<float>(m->theta);
        a.xi = static_cast<float>(m->xi);
        a.rho = static_cast<float>(m->rho);
        a.rhoc = static_cast<float>(std::sqrt(1.0 - m->rho * m->rho));
        a.K = K;
    }
    a.pay = ps;
    const int block = greeks_block();
    const int occ = greeks_occupancy(a.model, np);
    if (occ <= 0) return fail(MC_ECUDA, "Greeks kernel cannot be resident");
    int grid = 0, ppt = 1;
    size_grid(c->paths, block, occ * di.sms, &grid, &ppt);
    a.run.ppt = ppt;

    mc_plan P;  // owns the scratch buffers (freed on return)
    P.np = nv;
    MC_CUDA(dev_alloc(&P.partials, static_cast<size_t>(grid) * nv * 2 * sizeof(float)));
    MC_CUDA(dev_alloc(&P.ticket, sizeof(unsigned int)));
    MC_CUDA(cudaMemsetAsync(P.ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(dev_alloc(&P.dout, static_cast<size_t>(nv) * sizeof(mc_result)));
    if (m->kind == MC_HESTON) {
        const size_t nseg = (c->steps + K - 1) / K;
        MC_CUDA(dev_alloc(&P.ckpt, nseg * 2 * static_cast<size_t>(grid) * block * sizeof(float)));
    }
    a.ckpt = P.ckpt;
    a.red.partials = P.partials;
    a.red.ticket = P.ticket;
    a.red.out = P.dout;
    a.red.paths = c->paths;
    a.red.disc = std::exp(-m->r * c->T);
    a.red.err = nullptr;
    MC_CUDA(launch_greeks(a, grid, s));
    std::vector<mc_result> tmp(nv);
    MC_CUDA(cudaMemcpyAsync(tmp.data(), P.dout, nv * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    P.idle = true;
    for (int p = 0; p < np; ++p) {
        if (prices) prices[p] = tmp[static_cast<size_t>(p) * (G + 1)];
        for (int k = 0; k < G; ++k) greeks[static_cast<size_t>(p) * G + k] = tmp[static_cast<size_t>(p) * (G + 1) + 1 + k];
    }
    return MC_OK;
}

// mc_corr_greeks for kCorrMaxD < d <= kBigMaxD (arguments already checked):
// the per-path vectors in global memory, the contractions as FP32 products,
// the Cholesky adjoint of each batch in global memory (k_corr.cu).
static int corr_greeks_wide(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pay, mc_result *price,
                            mc_result *dl, mc_result *drho, cudaStream_t s, const DeviceInfo &di)
{
    const int d = m->d;
    const size_t dd = static_cast<size_t>(d) * d, tri = static_cast<size_t>(d) * (d + 1) / 2;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt), disc = std::exp(-m->r * c->T);
    const int64_t P = c->paths;
    if (P * d > (int64_t(1) << 31))
        return fail(MC_EUNSUPPORTED, "correlation sensitivities for d > %d hold paths x d <= 2^31 values per buffer",
                    kCorrMaxD);
    CorrArgs a{};
    a.run.paths = P;
    a.run.path_offset = c->path_offset;
    set_seed(a.run, c->seed);
    a.run.steps = c->steps;
    a.run.save_every = 1;
    a.d = d;
    a.exact4 = d % 4 == 0 ? 1 : 0;
    a.kind = pay->kind;
    a.strike = static_cast<float>(pay->strike);
    // batches of kchunk paths (a multiple of 16) for the batch-means errors
    int B = static_cast<int>(std::min<int64_t>(32, std::max<int64_t>(1, (P + 127) / 128)));
    const int kchunk = static_cast<int>(((P + B - 1) / B + 15) / 16 * 16);
    B = static_cast<int>((P + kchunk - 1) / kchunk);
    const int64_t uwarps = std::min<int64_t>(P, int64_t(1) << 20);
    const int ugrid = static_cast<int>((uwarps * 32 + 255) / 256);
    const int wgrid = static_cast<int>(std::min<int64_t>((P + 127) / 128, static_cast<int64_t>(di.sms) * 8));

    DeviceArena ar;
    const size_t bytes = DeviceArena::up(dd * 8) * 2 + DeviceArena::up(d * 8) * 2 + DeviceArena::up(sizeof(int)) +
                         DeviceArena::up(tri * 4) + DeviceArena::up(d * 4) * 2 + DeviceArena::up(dd * 4) +
                         DeviceArena::up(static_cast<size_t>(P) * d * 4) * 2 + DeviceArena::up(B * dd * 4) +
                         DeviceArena::up(B * 8) + 4 * DeviceArena::up((B + 1) * dd * 8) + DeviceArena::up(dd * 8) +
                         2 * DeviceArena::up(dd * sizeof(mc_result)) + DeviceArena::up(static_cast<size_t>(ugrid) * 2 * 4) +
                         DeviceArena::up(4) + DeviceArena::up(sizeof(mc_result));
    MC_CUDA(dev_alloc(&ar.base, bytes));
    double *dcorr = ar.take<double>(dd), *dL = ar.take<double>(dd), *dsig = ar.take<double>(d);
    double *dcfac = ar.take<double>(d);
    int *dstatus = ar.take<int>(1);
    float *dLp = ar.take<float>(tri), *ddrift = ar.take<float>(d), *dws0 = ar.take<float>(d), *dLs = ar.take<float>(dd);
    CorrWide w{};
    w.Wbuf = ar.take<float>(static_cast<size_t>(P) * d);
    w.Ybuf = ar.take<float>(static_cast<size_t>(P) * d);
    w.part = ar.take<float>(B * dd);
    double *dnb = ar.take<double>(B);
    w.Lt = ar.take<double>(dd);
    w.Pm = ar.take<double>((B + 1) * dd);
    w.Sm = ar.take<double>((B + 1) * dd);
    w.out_dl = ar.take<double>((B + 1) * dd);
    w.out_drho = ar.take<double>((B + 1) * dd);
    w.res_dl = ar.take<mc_result>(dd);
    w.res_drho = ar.take<mc_result>(dd);
    a.red.partials = ar.take<float>(static_cast<size_t>(ugrid) * 2);
    a.red.ticket = ar.take<unsigned int>(1);
    a.red.out = ar.take<mc_result>(1);
    a.red.paths = P;
    a.red.disc = disc;
    a.red.err = nullptr;
    w.Ls = dLs;
    w.drift = ddrift;
    w.ws0 = dws0;
    w.L = dL;
    w.cfac = dcfac;
    w.nb = dnb;
    w.batches = B;
    w.kchunk = kchunk;

    std::vector<double> corr(dd, 0.0), cf(d), nb(B);
    if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
    else for (int k = 0; k < d; ++k) corr[static_cast<size_t>(k) * d + k] = 1.0;
    for (int k = 0; k < d; ++k) cf[k] = disc * sdt * m->sigma[k];
    for (int b = 0; b < B; ++b) nb[b] = static_cast<double>(std::min<int64_t>(P, int64_t(b + 1) * kchunk) - int64_t(b) * kchunk);
    std::vector<float> ws0(d);
    for (int k = 0; k < d; ++k) ws0[k] = static_cast<float>((m->weights ? m->weights[k] : 1.0 / d) * m->s0[k]);
    MC_CUDA(cudaMemsetAsync(a.red.ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(cudaMemcpyAsync(dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dcfac, cf.data(), d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dnb, nb.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dws0, ws0.data(), d * sizeof(float), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_cholesky(d, dcorr, dL, dstatus, s));
    MC_CUDA(launch_scale_factor(d, dL, dsig, M_LOG2E, sdt, m->r, dt, MC_LOG_EULER, dLp, ddrift, s));
    int status = 0;
    MC_CUDA(cudaMemcpyAsync(&status, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    std::vector<float> Lp(tri), Ls(dd, 0.0f);
    MC_CUDA(cudaMemcpyAsync(Lp.data(), dLp, tri * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) Ls[static_cast<size_t>(i) * d + j] = Lp[static_cast<size_t>(i) * (i + 1) / 2 + j];
    MC_CUDA(cudaMemcpyAsync(dLs, Ls.data(), dd * sizeof(float), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_corr_wide(a, w, wgrid, s));
    mc_result pr;
    std::vector<mc_result> hdl(dd), hdr(dd);
    MC_CUDA(cudaMemcpyAsync(&pr, a.red.out, sizeof pr, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(hdl.data(), w.res_dl, dd * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(hdr.data(), w.res_drho, dd * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    ar.idle = true;
    if (price) *price = pr;
    if (dl) std::memcpy(dl, hdl.data(), dd * sizeof(mc_result));
    if (drho) std::memcpy(drho, hdr.data(), dd * sizeof(mc_result));
    return MC_OK;
}

int mc_corr_greeks(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pay, mc_result *price, mc_result *dl,
                   mc_result *drho, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_corr_greeks");
    int rc;
    if ((rc = check_model(m)) || (rc = check_cfg(c, m))) return rc;
    if (!pay) return fail(MC_EINVAL, "payoff is NULL");
    if (m->kind != MC_GBM || m->loadings || m->d < 2 || m->d > kBigMaxD)
        return fail(MC_EUNSUPPORTED, "correlation sensitivities: correlated GBM baskets with 2 <= d <= %d "
                                     "(Cholesky correlation)", kBigMaxD);
    if (c->scheme != MC_LOG_EULER) return fail(MC_EUNSUPPORTED, "correlation sensitivities use the log-Euler scheme");
    if (c->precision != MC_FP32) return fail(MC_EUNSUPPORTED, "correlation sensitivities are computed in FP32");
    if (c->monitoring != MC_DISCRETE) return fail(MC_EUNSUPPORTED, "correlation sensitivities: European payoffs only");
    const bool asian = pay->kind == MC_ASIAN_CALL || pay->kind == MC_ASIAN_PUT;
    if (pay->kind != MC_CALL && pay->kind != MC_PUT && !asian)
        return fail(MC_EUNSUPPORTED, "correlation sensitivities: a European or Asian basket call or put");
    if (asian && m->d > kCorrMaxD)
        return fail(MC_EUNSUPPORTED, "correlation sensitivities of Asian payoffs for d <= %d", kCorrMaxD);
    if (!std::isfinite(pay->strike)) return fail(MC_EINVAL, "strike not finite");
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m->d > kCorrMaxD) return corr_greeks_wide(m, c, pay, price, dl, drho, s, di);
    const int d = m->d;
    const size_t dd = static_cast<size_t>(d) * d;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt), disc = std::exp(-m->r * c->T);

    CorrArgs a{};
    a.run.paths = c->paths;
    a.run.path_offset = c->path_offset;
    set_seed(a.run, c->seed);
    a.run.steps = c->steps;
    a.run.save_every = 1;
    a.d = d;
    a.exact4 = d % 4 == 0 ? 1 : 0;
    a.kind = pay->kind;
    a.strike = static_cast<float>(pay->strike);
    const int occ = corr_occupancy(a);
    if (occ <= 0) return fail(MC_ECUDA, "correlation-sensitivity kernel cannot be resident");
    const int64_t tiles = (c->paths + corr_block() - 1) / corr_block();
    const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(occ) * di.sms));
    const int B = std::min(grid, 64);
    const size_t H = static_cast<size_t>(kCorrMaxD) * kCorrMaxD;

    DeviceArena ar;
    const size_t bytes = DeviceArena::up(dd * 8) * 2 + DeviceArena::up(d * 8) * 2 + DeviceArena::up(sizeof(int)) +
                         DeviceArena::up(static_cast<size_t>(grid) * H * 4) + DeviceArena::up(grid * 8) +
                         DeviceArena::up(static_cast<size_t>(B) * H * 8) + DeviceArena::up(B * 8) +
                         2 * DeviceArena::up((B + 1) * dd * 8) + 2 * DeviceArena::up(dd * sizeof(mc_result)) +
                         DeviceArena::up(static_cast<size_t>(grid) * 2 * 4) + DeviceArena::up(4) +
                         DeviceArena::up(sizeof(mc_result)) + DeviceArena::up(sizeof(float) * (kCorrMaxD * (kCorrMaxD + 1) / 2 + kCorrMaxD));
    MC_CUDA(dev_alloc(&ar.base, bytes));
    double *dcorr = ar.take<double>(dd), *dL = ar.take<double>(dd), *dsig = ar.take<double>(d);
    double *dcfac = ar.take<double>(d);
    int *dstatus = ar.take<int>(1);
    a.partials = ar.take<float>(static_cast<size_t>(grid) * H);
    a.counts = ar.take<double>(grid);
    double *Hb = ar.take<double>(static_cast<size_t>(B) * H), *nb = ar.take<double>(B);
    double *odl = ar.take<double>((B + 1) * dd), *odr = ar.take<double>((B + 1) * dd);
    mc_result *rdl = ar.take<mc_result>(dd), *rdr = ar.take<mc_result>(dd);
    a.red.partials = ar.take<float>(static_cast<size_t>(grid) * 2);
    a.red.ticket = ar.take<unsigned int>(1);
    a.red.out = ar.take<mc_result>(1);
    float *dLp = ar.take<float>(kCorrMaxD * (kCorrMaxD + 1) / 2 + kCorrMaxD), *ddrift = dLp + kCorrMaxD * (kCorrMaxD + 1) / 2;
    a.red.paths = c->paths;
    a.red.disc = disc;
    a.red.err = nullptr;

    std::vector<double> corr(dd, 0.0), cf(d);
    if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
    else for (int k = 0; k < d; ++k) corr[static_cast<size_t>(k) * d + k] = 1.0;
    for (int k = 0; k < d; ++k) cf[k] = disc * sdt * m->sigma[k];
    MC_CUDA(cudaMemsetAsync(a.red.ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(cudaMemcpyAsync(dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(dcfac, cf.data(), d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_cholesky(d, dcorr, dL, dstatus, s));
    MC_CUDA(launch_scale_factor(d, dL, dsig, M_LOG2E, sdt, m->r, dt, MC_LOG_EULER, dLp, ddrift, s));
    std::vector<float> Lp(static_cast<size_t>(d) * (d + 1) / 2), drift(d);
    int status = 0;
    MC_CUDA(cudaMemcpyAsync(&status, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(Lp.data(), dLp, Lp.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(drift.data(), ddrift, d * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    CorrConst k{};
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) k.L[i * (i + 1) / 2 + j] = Lp[static_cast<size_t>(i) * (i + 1) / 2 + j];
        k.drift[i] = drift[i];
        const double w = m->weights ? m->weights[i] : 1.0 / d;
        k.ws0[i] = static_cast<float>(w * m->s0[i]);
    }
    MC_CUDA(launch_corr(a, k, grid, B, dL, dcfac, Hb, nb, odl, odr, rdl, rdr, s));
    mc_result pr;
    std::vector<mc_result> hdl(dd), hdr(dd);
    MC_CUDA(cudaMemcpyAsync(&pr, a.red.out, sizeof pr, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(hdl.data(), rdl, dd * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(hdr.data(), rdr, dd * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    ar.idle = true;
    if (price) *price = pr;
    if (dl) std::memcpy(dl, hdl.data(), dd * sizeof(mc_result));
    if (drho) std::memcpy(drho, hdr.data(), dd * sizeof(mc_result));
    return MC_OK;
}

int mc_price_mlmc(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pays, int32_t np, int64_t paths_ref,
                  mc_mlmc_result *out, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_price_mlmc");
    int rc;
    if (!out) return fail(MC_EINVAL, "out is NULL");
    if ((rc = check_model(m)) || (rc = check_cfg(c, m))) return rc;
    if (m->kind != MC_GBM || m->d < 2 || m->d > 64 || m->loadings)
        return fail(MC_EUNSUPPORTED, "two-level precision estimator: correlated GBM baskets with 2 <= d <= 64 "
                                     "(Cholesky correlation)");
    if (c->precision == MC_FP32) return fail(MC_EINVAL, "the coarse level needs a reduced precision (BF16, FP16, E4M3)");
    if (c->monitoring != MC_DISCRETE) return fail(MC_EUNSUPPORTED, "two-level estimator: discrete monitoring only");
    if (np < 1 || np > kMlmcMaxPayoffs) return fail(MC_EINVAL, "n_payoff = %d outside [1, %d]", np, kMlmcMaxPayoffs);
    if (paths_ref < 2) return fail(MC_EINVAL, "paths_ref = %lld must be >= 2", static_cast<long long>(paths_ref));
    if (c->path_offset + c->paths + paths_ref > (int64_t(1) << 56)) return fail(MC_EINVAL, "path range must lie in [0, 2^56)");
    PayoffSet ps;
    if ((rc = build_payoffs(pays, np, &ps))) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // level 0: the reduced-precision tensor-core estimator on [offset, offset + N0)
    std::vector<mc_result> coarse(np);
    if ((rc = mc_price(m, c, pays, np, coarse.data(), stream))) return rc;

    // level 1: both arithmetics on the next paths_ref paths
    const int d = m->d;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const double cfac = c->scheme == MC_LOG_EULER ? M_LOG2E : 1.0;
    const size_t dd = static_cast<size_t>(d) * d, tri = static_cast<size_t>(d) * (d + 1) / 2;
    mc_plan P;  // owns the scratch buffers (freed on return)
    MC_CUDA(dev_alloc(&P.dcorr, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dL, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dsig, d * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dLp, (tri + 64 * 65 / 2 + 64) * sizeof(float)));
    MC_CUDA(dev_alloc(&P.ddrift, d * sizeof(float)));
    MC_CUDA(dev_alloc(&P.dstatus, sizeof(int)));
    std::vector<double> corr(dd, 0.0);
    if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
    else for (int a = 0; a < d; ++a) corr[static_cast<size_t>(a) * d + a] = 1.0;
    MC_CUDA(cudaMemcpyAsync(P.dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(P.dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_cholesky(d, P.dcorr, P.dL, P.dstatus, s));
    float *dLq = P.dLp + tri, *dcsq = dLq + 64 * 65 / 2;
    MC_CUDA(launch_scale_factor(d, P.dL, P.dsig, cfac, sdt, m->r, dt, c->scheme, P.dLp, P.ddrift, s));
    MC_CUDA(launch_mlmc_prep(c->precision, d, P.dL, P.dsig, cfac, sdt, dLq, dcsq, s));
    std::vector<float> Lp(tri), Lq(64 * 65 / 2), csq(64), drift(d);
    int status = 0;
    MC_CUDA(cudaMemcpyAsync(&status, P.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(Lp.data(), P.dLp, tri * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(Lq.data(), dLq, Lq.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(csq.data(), dcsq, 64 * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(drift.data(), P.ddrift, d * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    MlmcConst k;
    std::memset(&k, 0, sizeof k);
    float *kL = reinterpret_cast<float *>(k.Lp), *kLq = reinterpret_cast<float *>(k.Lqp);
    for (int a = 0; a < 64; ++a) {
        for (int j = 0; j <= a; ++j) {  // row a of column j: pair a / 2 of the column's run, lane a & 1
            const int e = 2 * (basket_pair_base(64, j) + a / 2 - j / 2) + (a & 1);
            kL[e] = a < d ? Lp[static_cast<size_t>(a) * (a + 1) / 2 + j] : 0.0f;
            kLq[e] = Lq[a * (a + 1) / 2 + j];
        }
        k.csq[a] = csq[a];
        if (a < d) {
            const double w = m->weights ? m->weights[a] : 1.0 / d;
            k.drift[a] = drift[a];
            k.ws0[a] = static_cast<float>(w * m->s0[a]);
            k.w[a] = static_cast<float>(w);
            k.s0[a] = static_cast<float>(m->s0[a]);
        } else {
            k.s0[a] = 1.0f;  // padded columns: zero weight, inert state
        }
    }
    MlmcArgs a{};
    a.run.paths = paths_ref;
    a.run.path_offset = c->path_offset + c->paths;
    set_seed(a.run, c->seed);
    a.run.steps = c->steps;
    a.run.save_every = 1;
    a.d = d;
    a.scheme = c->scheme;
    a.pay = ps;
    const int nv = 3 * np;
    const int occ = mlmc_occupancy(c->precision, a);
    if (occ <= 0) return fail(MC_ECUDA, "correction kernel cannot be resident");
    int grid = 0, ppt = 1;
    size_grid(paths_ref, mlmc_paths_per_block(), occ * di.sms, &grid, &ppt);
    a.run.ppt = ppt;
    MC_CUDA(dev_alloc(&P.partials, static_cast<size_t>(grid) * nv * 2 * sizeof(float)));
    MC_CUDA(dev_alloc(&P.ticket, sizeof(unsigned int)));
    MC_CUDA(cudaMemsetAsync(P.ticket, 0, sizeof(unsigned int), s));
    MC_CUDA(dev_alloc(&P.dout, static_cast<size_t>(nv) * sizeof(mc_result)));
    a.red.partials = P.partials;
    a.red.ticket = P.ticket;
    a.red.out = P.dout;
    a.red.paths = paths_ref;
    a.red.disc = std::exp(-m->r * c->T);
    a.red.err = nullptr;
    MC_CUDA(launch_mlmc_coupled(c->precision, a, k, grid, s));
    std::vector<mc_result> lv(nv);
    MC_CUDA(cudaMemcpyAsync(lv.data(), P.dout, nv * sizeof(mc_result), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    P.idle = true;
    for (int p = 0; p < np; ++p) {
        mc_mlmc_result &o = out[p];
        o.coarse = coarse[p];
        o.correction = lv[p];
        o.ref_level = lv[np + p];
        o.coarse_level = lv[2 * np + p];
        o.price = coarse[p].price + lv[p].price;
        o.se = std::sqrt(coarse[p].se * coarse[p].se + lv[p].se * lv[p].se);
    }
    return MC_OK;
}

int mc_price_qmc(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *pays, int32_t np, int32_t reps,
                 mc_result *out, double *rep_means, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_price_qmc");
    int rc;
    if (!out) return fail(MC_EINVAL, "out is NULL");
    if ((rc = check_model(m)) || (rc = check_cfg(c, m))) return rc;
    if (m->kind != MC_GBM || m->d > kQmcMaxAssets || m->loadings)
        return fail(MC_EUNSUPPORTED, "quasi-Monte Carlo: GBM with d <= %d (Cholesky correlation)", kQmcMaxAssets);
    if (2 * m->d * c->steps > kQmcMaxDims)
        return fail(MC_EUNSUPPORTED, "quasi-Monte Carlo: 2 d steps = %d exceeds %d Sobol dimensions",
                    2 * m->d * c->steps, kQmcMaxDims);
    if (c->precision != MC_FP32 || c->monitoring != MC_DISCRETE)
        return fail(MC_EUNSUPPORTED, "quasi-Monte Carlo: FP32 contraction and discrete monitoring");
    if (c->path_offset + c->paths > (int64_t(1) << 23))
        return fail(MC_EINVAL, "quasi-Monte Carlo: points must lie in [0, 2^23) (23-bit uniforms)");
    if (reps < 2 || reps > 65535) return fail(MC_EINVAL, "replications = %d outside [2, 65535]", reps);
    if (np < 1) return fail(MC_EINVAL, "n_payoff must be >= 1");
    PayoffSet ps;
    if ((rc = build_payoffs(pays, np, &ps))) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const int d = m->d;
    const double dt = c->T / c->steps, sdt = std::sqrt(dt);
    const double cfac = c->scheme == MC_LOG_EULER ? M_LOG2E : 1.0;
    const size_t dd = static_cast<size_t>(d) * d, tri = static_cast<size_t>(d) * (d + 1) / 2;
    mc_plan P;  // owns the scratch buffers (freed on return)
    MC_CUDA(dev_alloc(&P.dcorr, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dL, dd * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dsig, d * sizeof(double)));
    MC_CUDA(dev_alloc(&P.dLp, tri * sizeof(float)));
    MC_CUDA(dev_alloc(&P.ddrift, d * sizeof(float)));
    MC_CUDA(dev_alloc(&P.dstatus, sizeof(int)));
    std::vector<double> corr(dd, 0.0);
    if (m->corr) std::memcpy(corr.data(), m->corr, dd * sizeof(double));
    else for (int a = 0; a < d; ++a) corr[static_cast<size_t>(a) * d + a] = 1.0;
    MC_CUDA(cudaMemcpyAsync(P.dcorr, corr.data(), dd * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(P.dsig, m->sigma, d * sizeof(double), cudaMemcpyHostToDevice, s));
    MC_CUDA(launch_cholesky(d, P.dcorr, P.dL, P.dstatus, s));
    MC_CUDA(launch_scale_factor(d, P.dL, P.dsig, cfac, sdt, m->r, dt, c->scheme, P.dLp, P.ddrift, s));
    std::vector<float> Lp(tri), drift(d);
    int status = 0;
    MC_CUDA(cudaMemcpyAsync(&status, P.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(Lp.data(), P.dLp, tri * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(drift.data(), P.ddrift, d * sizeof(float), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (status) return fail(MC_ENOTPSD, "correlation matrix is not positive definite");
    QmcConst k;
    std::memset(&k, 0, sizeof k);
    const int ndim = 2 * d * c->steps;
    qmc_directions(ndim, k.V);
    for (int a = 0; a < kQmcMaxAssets; ++a) {
        if (a < d) {
            for (int j = 0; j <= a; ++j) k.L[a * (a + 1) / 2 + j] = Lp[static_cast<size_t>(a) * (a + 1) / 2 + j];
            const double w = m->weights ? m->weights[a] : 1.0 / d;
            k.drift[a] = drift[a];
            k.ws0[a] = static_cast<float>(w * m->s0[a]);
            k.w[a] = static_cast<float>(w);
            k.s0[a] = static_cast<float>(m->s0[a]);
        } else {
            k.s0[a] = 1.0f;  // padded columns: zero weight, inert state
        }
    }
    QmcArgs a{};
    a.n0 = c->path_offset;
    a.npts = c->paths;
    a.steps = c->steps;
    a.d = d;
    a.scheme = c->scheme;
    a.ndim = ndim;
    a.reps = reps;
    a.k0 = static_cast<uint32_t>(c->seed);
    a.k1 = static_cast<uint32_t>(c->seed >> 32);
    a.rk = round_keys(a.k0, a.k1);
    a.pay = ps;
    MC_CUDA(dev_alloc(&P.dsums, static_cast<size_t>(reps) * np * sizeof(double)));
    MC_CUDA(cudaMemsetAsync(P.dsums, 0, static_cast<size_t>(reps) * np * sizeof(double), s));
    a.sums = P.dsums;
    const int occ = qmc_occupancy(a);
    if (occ <= 0) return fail(MC_ECUDA, "quasi-Monte Carlo kernel cannot be resident");
    const int64_t blocks = (c->paths + qmc_block() - 1) / qmc_block();
    const int64_t per_rep = std::max<int64_t>(1, static_cast<int64_t>(occ) * di.sms / reps);
    const int grid = static_cast<int>(std::min<int64_t>(blocks, std::max<int64_t>(per_rep, 1)));
    MC_CUDA(launch_qmc(a, k, grid, s));
    std::vector<double> sums(static_cast<size_t>(reps) * np);
    MC_CUDA(cudaMemcpyAsync(sums.data(), P.dsums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    P.idle = true;
    const double disc = std::exp(-m->r * c->T), N = static_cast<double>(c->paths);
    for (int p = 0; p < np; ++p) {
        double mean = 0.0, m2 = 0.0;
        for (int r = 0; r < reps; ++r) {
            const double v = disc * sums[static_cast<size_t>(r) * np + p] / N;
            if (rep_means) rep_means[static_cast<size_t>(r) * np + p] = v;
            mean += v;
        }
        mean /= reps;
        for (int r = 0; r < reps; ++r) {
            const double v = disc * sums[static_cast<size_t>(r) * np + p] / N - mean;
            m2 += v * v;
        }
        out[p].price = mean;
        out[p].se = std::sqrt(m2 / (reps - 1) / reps);
    }
    return MC_OK;
}

int mc_simulate(const mc_model *model, const mc_sim_cfg *cfg, int32_t save_every, float *dev_out, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_simulate");
    if (!dev_out) return fail(MC_EINVAL, "dev_out is NULL");
    if (!cfg) return fail(MC_EINVAL, "cfg is NULL");
    if (save_every < 1 || cfg->steps < 1 || cfg->steps % save_every)
        return fail(MC_EINVAL, "save_every = %d must divide steps = %d", save_every, cfg ? cfg->steps : 0);
    mc_plan P;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = plan_setup(&P, model, cfg, nullptr, 0, dev_out, save_every, s);
    if (rc) return rc;
    rc = plan_launch(&P, nullptr, s);
    if (rc) return rc;
    // P's set-up buffers are released when it goes out of scope; the kernel
    // no longer needs them (the factor travels in the launch parameters), but
    // cudaFree must not race the launch's argument capture: synchronise.
    MC_CUDA(cudaStreamSynchronize(s));
    P.idle = true;
    return MC_OK;
}

}  // extern "C"
