// mc_price_gbm1d_noalloc: the single-asset GBM pricer for callers that must
// not allocate device memory (for example code running inside another
// framework's memory pool or allocator hooks, or code whose allocations are
// forbidden while a graph or a real-time loop is being driven).  It launches
// the same kernel as mc_price, but the kernel's scratch (one FP32 partial-sum
// pair per block and payoff, and the last-block ticket) lives in the
// file-scope device array below instead of memory from cudaMalloc.  The
// caller passes the output buffer; nothing is allocated or freed.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "mc_kernels.cuh"

namespace {

// Capacity: 256 bytes for the ticket, then MC_NOALLOC_PARTIALS floats of
// per-block partial sums (2 per payoff per block).  Every GPU that loads the
// library holds this array (about 512 KiB) until the process exits.
constexpr size_t kTicketBytes = 256;
constexpr size_t kPartialFloats = MC_NOALLOC_PARTIALS;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kTicketBytes + kPartialFloats * sizeof(float)];

// Device address of g_noalloc_scratch per device, resolved once with that
// device current (the host-side name of a __device__ variable is only a
// stand-in, never a device address).
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int noalloc_fail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return gbmc::set_last_error(code, buf);
}

int scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MC_EUNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(MC_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return MC_OK;
}

}  // namespace

extern "C" int mc_price_gbm1d_noalloc(const mc_model *m, const mc_sim_cfg *c, const mc_payoff *p,
                                      int32_t n_payoff, mc_result *dev_out, void *stream)
{
    using namespace gbmc;
    if (!dev_out) return noalloc_fail(MC_EINVAL, "dev_out is NULL");
    if (n_payoff < 1 || n_payoff > MC_MAX_PAYOFFS)
        return noalloc_fail(MC_EINVAL, "n_payoff = %d outside [1, %d]", n_payoff, MC_MAX_PAYOFFS);
    // The same checks as mc_price (finite and positive s0, sigma, T; finite
    // r, weights, strikes; no NaN barrier; path range inside [0, 2^56);
    // unit correlation diagonal), then this entry point's own restrictions.
    PayoffSet ps{};
    int rc = check_price_args(m, c, p, n_payoff, &ps);
    if (rc) return rc;
    if (m->kind != MC_GBM || m->d != 1 || m->loadings)
        return noalloc_fail(MC_EINVAL, "single-asset GBM only (kind MC_GBM, d = 1, no loadings)");
    if (m->corr && std::fabs(m->corr[0] - 1.0) > 1e-12) return noalloc_fail(MC_EINVAL, "corr[0] must be 1");
    if (c->monitoring != MC_DISCRETE) return noalloc_fail(MC_EUNSUPPORTED, "discrete barrier monitoring only");

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return noalloc_fail(MC_ECUDA, "device query: %s", cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    rc = scratch_for_device(dev, &scratch);
    if (rc) return rc;

    const double dt = c->T / c->steps, sdt = std::sqrt(dt), sg = m->sigma[0];
    const double w = m->weights ? m->weights[0] : 1.0;
    Gbm1dArgs a{};
    a.run.paths = c->paths;
    a.run.path_offset = c->path_offset;
    set_seed(a.run, c->seed);
    a.run.steps = c->steps;
    a.run.save = nullptr;
    a.run.save_every = 1;
    a.scheme = c->scheme;
    a.s0 = static_cast<float>(w * m->s0[0]);
    if (c->scheme == MC_LOG_EULER) {
        a.a = static_cast<float>(M_LOG2E * (m->r - 0.5 * sg * sg) * dt);
        a.b = static_cast<float>(M_LOG2E * sg * sdt);
    } else {
        a.a = static_cast<float>(m->r * dt);
        a.b = static_cast<float>(sg * sdt);
    }
    a.pay = ps;

    // Grid: one resident wave, and no more blocks than the partial-sum
    // capacity holds for this payoff count.
    const int block = 256;
    const int occ = gbm1d_occupancy(a, block);
    if (occ <= 0) return noalloc_fail(MC_ECUDA, "occupancy query failed");
    int64_t grid = static_cast<int64_t>(occ) * sms;
    const int64_t cap_blocks = static_cast<int64_t>(kPartialFloats) / (2 * n_payoff);
    if (grid > cap_blocks) grid = cap_blocks;
    const int64_t need = (c->paths + block - 1) / block;
    if (grid > need) grid = need;
    const int64_t ppt = (c->paths + grid * block - 1) / (grid * block);
    grid = (c->paths + ppt * block - 1) / (ppt * block);
    if (ppt > INT32_MAX) return noalloc_fail(MC_EINVAL, "paths too large for one launch");
    a.run.ppt = static_cast<int>(ppt);

    a.red.ticket = reinterpret_cast<unsigned int *>(scratch);
    a.red.partials = reinterpret_cast<float *>(scratch + kTicketBytes);
    a.red.out = dev_out;
    a.red.paths = c->paths;
    a.red.disc = std::exp(-m->r * c->T);
    a.red.err = nullptr;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The ticket must start at zero; a previous call leaves it at zero, but
    // an interrupted one might not.  (Memset allocates nothing.)
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = launch_gbm1d(a, static_cast<int>(grid), block, s);
    if (e != cudaSuccess) return noalloc_fail(MC_ECUDA, "launch: %s", cudaGetErrorString(e));
    return MC_OK;
}
