// C ABI of the surrogate network (mc_mlp_* in include/mc.h): parameter
// storage, forward evaluation, loss/gradient, and the native training loop
// (mini-batch Adam) that drives the kernels of k_mlp.cu.
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "mc_kernels.cuh"
#include "mlp.cuh"

using namespace gbmc;

struct mc_mlp {
    MlpLayout L;
    int device = -1;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *work = nullptr;
    size_t work_floats = 0;
    double *partial = nullptr;
    double *dpartial = nullptr;  // loss parts of the derivative-label loss, (1 + kMlpMaxDirs) x kPartials
    int step = 0;
    // bf16 operand image of the weights, rebuilt when the parameters change
    uint8_t *img = nullptr;
    uint64_t version = 1, img_version = 0;
    unsigned int *err = nullptr;  // set by the bf16 kernel when a bounded wait expires
    int train_mode = MC_MLP_TRAIN_FP32;  // arithmetic of mc_mlp_loss_grad / mc_mlp_train
    ~mc_mlp()
    {
        for (float *p : {params, grad, m, v, work})
            if (p) cudaFree(p);
        if (partial) cudaFree(partial);
        if (dpartial) cudaFree(dpartial);
        if (img) cudaFree(img);
        if (err) cudaFree(err);
    }
};

namespace {

constexpr int kPartials = 512;

#define MLP_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            char b_[256];                                                                     \
            std::snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));           \
            return set_last_error(e_ == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA, b_); \
        }                                                                                     \
    } while (0)

int ensure_work(mc_mlp *N, size_t floats)
{
    if (N->work_floats >= floats) return MC_OK;
    if (N->work) cudaFree(N->work);
    N->work = nullptr;
    N->work_floats = 0;
    MLP_CUDA(cudaMalloc(&N->work, floats * sizeof(float)));
    N->work_floats = floats;
    return MC_OK;
}

// One batch's loss partials and gradient in the network's training arithmetic.
int loss_grad_batch(mc_mlp *N, const float *x, const float *t, int64_t n, cudaStream_t s)
{
    if (N->train_mode == MC_MLP_TRAIN_TF32X3) {
        if (!N->err) {
            MLP_CUDA(cudaMalloc(&N->err, sizeof(unsigned int)));
            MLP_CUDA(cudaMemsetAsync(N->err, 0, sizeof(unsigned int), s));
        }
        MLP_CUDA(mlp_loss_grad_tc(N->L, N->params, x, t, n, N->work, N->grad, N->partial, kPartials, N->err,
                                  mbar_wait_cap(), s));
    } else {
        MLP_CUDA(mlp_loss_grad(N->L, N->params, x, t, n, N->work, N->grad, N->partial, kPartials, s));
    }
    return MC_OK;
}

// Checks of a derivative-label loss description against the network.
int check_dloss(const mc_mlp *N, const mc_mlp_dloss *dl)
{
    if (!dl) return set_last_error(MC_EINVAL, "dloss is NULL");
    if (dl->n_dir < 0 || dl->n_dir > kMlpMaxDirs) return set_last_error(MC_EINVAL, "n_dir outside [0, 4]");
    if (N->L.sizes.size() < 3) return set_last_error(MC_EUNSUPPORTED, "derivative labels need a hidden layer");
    for (int k = 0; k < dl->n_dir; ++k) {
        if (dl->dir[k] < 0 || dl->dir[k] >= N->L.sizes[0]) return set_last_error(MC_EINVAL, "dir outside the inputs");
        if (!std::isfinite(dl->scale[k]) || !std::isfinite(dl->weight[k]) || dl->weight[k] < 0.0f)
            return set_last_error(MC_EINVAL, "scale must be finite and weight finite and >= 0");
    }
    return MC_OK;
}

// One batch of the derivative-label loss: loss parts at dpartial, gradient at grad.
int loss_grad_batch_d(mc_mlp *N, const float *x, const float *t, const float *g, int64_t n, const mc_mlp_dloss *dl,
                      cudaStream_t s)
{
    if (!N->dpartial) MLP_CUDA(cudaMalloc(&N->dpartial, (1 + kMlpMaxDirs) * kPartials * sizeof(double)));
    if (N->train_mode == MC_MLP_TRAIN_TF32X3) {
        if (!N->err) {
            MLP_CUDA(cudaMalloc(&N->err, sizeof(unsigned int)));
            MLP_CUDA(cudaMemsetAsync(N->err, 0, sizeof(unsigned int), s));
        }
        MLP_CUDA(mlp_loss_grad_d_tc(N->L, N->params, x, t, g, n, dl->n_dir, dl->dir, dl->scale, dl->weight, N->work,
                                    N->grad, N->dpartial, kPartials, N->err, mbar_wait_cap(), s));
    } else {
        MLP_CUDA(mlp_loss_grad_d(N->L, N->params, x, t, g, n, dl->n_dir, dl->dir, dl->scale, dl->weight, N->work,
                                 N->grad, N->dpartial, kPartials, s));
    }
    return MC_OK;
}

size_t train_floats_d(const mc_mlp *N, int64_t n, int K)
{
    return N->train_mode == MC_MLP_TRAIN_TF32X3 ? mlp_train_floats_d_tc(N->L, n, K) : mlp_train_floats_d(N->L, n, K);
}

size_t train_floats(const mc_mlp *N, int64_t n)
{
    return N->train_mode == MC_MLP_TRAIN_TF32X3 ? mlp_train_floats_tc(N->L, n) : mlp_train_floats(N->L, n);
}

int check_net(const mc_mlp *N)
{
    if (!N) return set_last_error(MC_EINVAL, "network is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != N->device)
        return set_last_error(MC_EINVAL, "network belongs to another device");
    return MC_OK;
}

}  // namespace

namespace gbmc {
const MlpLayout &mlp_layout_of(const mc_mlp *net) { return net->L; }

// Forward evaluation used by mc_risk (x, y device, n rows) on `s`.
int mlp_forward_any(mc_mlp *net, const float *x, int64_t n, float *y, int precision, cudaStream_t s)
{
    return mc_mlp_forward(net, x, n, y, precision, s);
}

// Reads and clears the tensor-core kernels' time-out word (synchronises `s`).
int mlp_check_timeout(mc_mlp *net, cudaStream_t s)
{
    if (!net->err) return MC_OK;
    unsigned int e = 0;
    MLP_CUDA(cudaMemcpyAsync(&e, net->err, sizeof e, cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaStreamSynchronize(s));
    if (!e) return MC_OK;
    MLP_CUDA(cudaMemsetAsync(net->err, 0, sizeof(unsigned int), s));
    return set_last_error(MC_ETIMEOUT, "a bounded wait of a tensor-core network kernel expired (outputs are NaN "
                                        "or undefined)");
}
}  // namespace gbmc

extern "C" {

int mc_mlp_create(int32_t n_in, int32_t width, int32_t hidden, const float *init, mc_mlp **out)
{
    if (!out) return set_last_error(MC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || width < 1 || width > 1024 || hidden < 1 || hidden > 16)
        return set_last_error(MC_EINVAL, "n_in in [1,64], width in [1,1024], hidden in [1,16]");
    if (!init) return set_last_error(MC_EINVAL, "init is NULL");
    mc_mlp *N = new (std::nothrow) mc_mlp();
    if (!N) return set_last_error(MC_ENOMEM, "host allocation failed");
    N->L = MlpLayout(n_in, width, hidden);
    const size_t bytes = static_cast<size_t>(N->L.count) * sizeof(float);
    auto fail_free = [&](int code) { delete N; return code; };
    if (cudaGetDevice(&N->device) != cudaSuccess) return fail_free(set_last_error(MC_ECUDA, "no device"));
    for (float **p : {&N->params, &N->grad, &N->m, &N->v})
        if (cudaMalloc(p, bytes) != cudaSuccess) return fail_free(set_last_error(MC_ENOMEM, "device allocation failed"));
    if (cudaMalloc(&N->partial, kPartials * sizeof(double)) != cudaSuccess)
        return fail_free(set_last_error(MC_ENOMEM, "device allocation failed"));
    if (cudaMemcpy(N->params, init, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(N->m, 0, bytes) != cudaSuccess || cudaMemset(N->v, 0, bytes) != cudaSuccess)
        return fail_free(set_last_error(MC_ECUDA, "initialisation copy failed"));
    *out = N;
    return MC_OK;
}

int64_t mc_mlp_param_count(const mc_mlp *net) { return net ? net->L.count : -1; }

int mc_mlp_get_params(const mc_mlp *net, float *host)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!host) return set_last_error(MC_EINVAL, "host is NULL");
    MLP_CUDA(cudaMemcpy(host, net->params, net->L.count * sizeof(float), cudaMemcpyDeviceToHost));
    return MC_OK;
}

int mc_mlp_set_params(mc_mlp *net, const float *host)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!host) return set_last_error(MC_EINVAL, "host is NULL");
    MLP_CUDA(cudaMemcpy(net->params, host, net->L.count * sizeof(float), cudaMemcpyHostToDevice));
    ++net->version;
    net->step = 0;
    MLP_CUDA(cudaMemset(net->m, 0, net->L.count * sizeof(float)));
    MLP_CUDA(cudaMemset(net->v, 0, net->L.count * sizeof(float)));
    return MC_OK;
}

int mc_mlp_forward(mc_mlp *net, const float *dev_x, int64_t n, float *dev_y, int32_t precision, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_mlp_forward");
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!dev_x || !dev_y || n < 1) return set_last_error(MC_EINVAL, "x, y must be set and n >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == MC_BF16) {
        if (!mlp_bf16_supported(net->L))
            return set_last_error(MC_EUNSUPPORTED, "bf16 inference needs n_in <= 10 and equal hidden widths, a "
                                                   "multiple of 32 up to 256");
        if (!net->img) MLP_CUDA(cudaMalloc(&net->img, mlp_bf16_image_bytes(net->L)));
        if (!net->err) {
            MLP_CUDA(cudaMalloc(&net->err, sizeof(unsigned int)));
            MLP_CUDA(cudaMemset(net->err, 0, sizeof(unsigned int)));
        }
        if (net->img_version != net->version) {
            MLP_CUDA(mlp_bf16_prepare(net->L, net->params, net->img, s));
            net->img_version = net->version;
        }
        MLP_CUDA(mlp_forward_bf16(net->L, net->params, net->img, dev_x, n, dev_y, net->err, mbar_wait_cap(), s));
        return MC_OK;
    }
    if (precision != MC_FP32) return set_last_error(MC_EUNSUPPORTED, "precision: MC_FP32 or MC_BF16");
    int maxw = 0;
    for (int v : net->L.sizes) maxw = v > maxw ? v : maxw;
    if ((rc = ensure_work(net, 2 * static_cast<size_t>(n < kMlpForwardSlice ? n : kMlpForwardSlice) * maxw))) return rc;
    MLP_CUDA(mlp_forward_fp32(net->L, net->params, dev_x, n, net->work, dev_y, s));
    return MC_OK;
}

int mc_mlp_loss_grad(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, double *loss, float *host_grad,
                     void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_mlp_loss_grad");
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!dev_x || !dev_t || n < 1) return set_last_error(MC_EINVAL, "x, t must be set and n >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_work(net, train_floats(net, n)))) return rc;
    if ((rc = loss_grad_batch(net, dev_x, dev_t, n, s))) return rc;
    std::vector<double> part(kPartials);
    MLP_CUDA(cudaMemcpyAsync(part.data(), net->partial, kPartials * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (host_grad)
        MLP_CUDA(cudaMemcpyAsync(host_grad, net->grad, net->L.count * sizeof(float), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (double p : part) tot += p;
    if (loss) *loss = tot / static_cast<double>(n);
    return mlp_check_timeout(net, s);
}

int mc_mlp_train(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, int32_t epochs, int32_t batch,
                 float lr, double *last_epoch_loss, void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_mlp_train");
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!dev_x || !dev_t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
        return set_last_error(MC_EINVAL, "x, t set; n, epochs, batch >= 1; lr > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t B = batch < n ? batch : n;
    if ((rc = ensure_work(net, train_floats(net, B)))) return rc;
    const int n_in = net->L.sizes[0];
    ++net->version;
    std::vector<double> part(kPartials);
    double epoch_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        epoch_loss = 0.0;
        const bool last = ep == epochs - 1;
        for (int64_t b0 = 0; b0 + B <= n; b0 += B) {  // whole batches; the samples are i.i.d.
            if ((rc = loss_grad_batch(net, dev_x + b0 * n_in, dev_t + b0, B, s))) return rc;
            MLP_CUDA(mlp_adam(net->L.count, net->params, net->grad, net->m, net->v, lr, ++net->step, s));
            if (last) {
                MLP_CUDA(cudaMemcpyAsync(part.data(), net->partial, kPartials * sizeof(double), cudaMemcpyDeviceToHost, s));
                MLP_CUDA(cudaStreamSynchronize(s));
                for (double p : part) epoch_loss += p;
            }
        }
    }
    MLP_CUDA(cudaStreamSynchronize(s));
    if (last_epoch_loss) *last_epoch_loss = epoch_loss / static_cast<double>((n / B) * B);
    return mlp_check_timeout(net, s);
}

int mc_mlp_set_train_mode(mc_mlp *net, int32_t mode)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (mode != MC_MLP_TRAIN_FP32 && mode != MC_MLP_TRAIN_TF32X3)
        return set_last_error(MC_EINVAL, "mode: MC_MLP_TRAIN_FP32 or MC_MLP_TRAIN_TF32X3");
    if (mode == MC_MLP_TRAIN_TF32X3 && !mlp_tc_supported(net->L))
        return set_last_error(MC_EUNSUPPORTED, "tensor-core training needs >= 2 hidden layers of a width that is a "
                                               "multiple of 64");
    net->train_mode = mode;
    return MC_OK;
}

int mc_mlp_apply_grad(mc_mlp *net, const float *host_grad, float lr, void *stream)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!host_grad || !(lr > 0.0f)) return set_last_error(MC_EINVAL, "host_grad set and lr > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MLP_CUDA(cudaMemcpyAsync(net->grad, host_grad, net->L.count * sizeof(float), cudaMemcpyHostToDevice, s));
    MLP_CUDA(mlp_adam(net->L.count, net->params, net->grad, net->m, net->v, lr, ++net->step, s));
    ++net->version;
    MLP_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

int mc_mlp_loss_grad_d(mc_mlp *net, const float *dev_x, const float *dev_t, const float *dev_g, int64_t n,
                       const mc_mlp_dloss *dl, double *loss_parts, float *host_grad, void *stream)
{
    int rc;
    if ((rc = check_net(net)) || (rc = check_dloss(net, dl))) return rc;
    if (!dev_x || !dev_t || (dl->n_dir > 0 && !dev_g) || n < 1)
        return set_last_error(MC_EINVAL, "x, t (and g with directions) must be set and n >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_work(net, train_floats_d(net, n, dl->n_dir)))) return rc;
    if ((rc = loss_grad_batch_d(net, dev_x, dev_t, dev_g, n, dl, s))) return rc;
    std::vector<double> part((1 + kMlpMaxDirs) * kPartials);
    MLP_CUDA(cudaMemcpyAsync(part.data(), net->dpartial, (1 + dl->n_dir) * kPartials * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    if (host_grad)
        MLP_CUDA(cudaMemcpyAsync(host_grad, net->grad, net->L.count * sizeof(float), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaStreamSynchronize(s));
    if ((rc = mlp_check_timeout(net, s))) return rc;
    if (loss_parts)
        for (int k = 0; k <= dl->n_dir; ++k) {
            double tot = 0.0;
            for (int b = 0; b < kPartials; ++b) tot += part[static_cast<size_t>(k) * kPartials + b];
            loss_parts[k] = tot / static_cast<double>(n);
        }
    return MC_OK;
}

int mc_mlp_train_d(mc_mlp *net, const float *dev_x, const float *dev_t, const float *dev_g, int64_t n,
                   const mc_mlp_dloss *dl, int32_t epochs, int32_t batch, float lr, double *last_epoch_loss,
                   void *stream)
{
    gbmc::NvtxRange nvtx_("gbmc: mc_mlp_train_d");
    int rc;
    if ((rc = check_net(net)) || (rc = check_dloss(net, dl))) return rc;
    if (!dev_x || !dev_t || (dl->n_dir > 0 && !dev_g) || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
        return set_last_error(MC_EINVAL, "x, t (and g) set; n, epochs, batch >= 1; lr > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t B = batch < n ? batch : n;
    if ((rc = ensure_work(net, train_floats_d(net, B, dl->n_dir)))) return rc;
    const int n_in = net->L.sizes[0], K = dl->n_dir;
    ++net->version;
    std::vector<double> part((1 + kMlpMaxDirs) * kPartials);
    double epoch_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        epoch_loss = 0.0;
        const bool last = ep == epochs - 1;
        for (int64_t b0 = 0; b0 + B <= n; b0 += B) {  // whole batches; the samples are i.i.d.
            if ((rc = loss_grad_batch_d(net, dev_x + b0 * n_in, dev_t + b0, K ? dev_g + b0 * K : nullptr, B, dl, s)))
                return rc;
            MLP_CUDA(mlp_adam(net->L.count, net->params, net->grad, net->m, net->v, lr, ++net->step, s));
            if (last) {
                MLP_CUDA(cudaMemcpyAsync(part.data(), net->dpartial, (1 + K) * kPartials * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
                MLP_CUDA(cudaStreamSynchronize(s));
                for (int k = 0; k < (1 + K) * kPartials; ++k) epoch_loss += part[k];
            }
        }
    }
    MLP_CUDA(cudaStreamSynchronize(s));
    if ((rc = mlp_check_timeout(net, s))) return rc;
    if (last_epoch_loss) *last_epoch_loss = epoch_loss / static_cast<double>((n / B) * B);
    return MC_OK;
}

int mc_mlp_loss_grad_sums(mc_mlp *net, const float *dev_x, const float *dev_t, int64_t n, float *dev_out,
                          void *stream)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!dev_x || !dev_t || !dev_out || n < 1) return set_last_error(MC_EINVAL, "x, t, out must be set and n >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_work(net, train_floats(net, n)))) return rc;
    if ((rc = loss_grad_batch(net, dev_x, dev_t, n, s))) return rc;
    MLP_CUDA(mlp_sums_out(net->L.count, net->grad, static_cast<double>(n), net->partial, kPartials, dev_out, s));
    return MC_OK;
}

int mc_mlp_apply_grad_sums(mc_mlp *net, const float *dev_grad, float scale, float lr, void *stream)
{
    int rc;
    if ((rc = check_net(net))) return rc;
    if (!dev_grad || !(lr > 0.0f) || !(scale > 0.0f) || !std::isfinite(scale))
        return set_last_error(MC_EINVAL, "dev_grad set, lr > 0 and a finite scale > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MLP_CUDA(mlp_scale_copy(net->L.count, dev_grad, scale, net->grad, s));
    MLP_CUDA(mlp_adam(net->L.count, net->params, net->grad, net->m, net->v, lr, ++net->step, s));
    ++net->version;
    return MC_OK;
}

int mc_mlp_destroy(mc_mlp *net)
{
    delete net;
    return MC_OK;
}

}  // extern "C"
