// Surrogate network: packed FP32 parameter layout and the device routines of
// k_mlp.cu / k_mlp_tc.cu used by the mc_mlp_* entry points and mc_risk.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace gbmc {

// Layer sizes n_in, width x hidden, 1; layer l's W_l [in x out] (row-major)
// at w_off[l], b_l [out] at b_off[l] in one packed FP32 vector.
struct MlpLayout {
    std::vector<int> sizes;
    std::vector<int64_t> w_off, b_off;
    int64_t count = 0;
    MlpLayout() = default;
    MlpLayout(int n_in, int width, int hidden);
};

// y[n] = net(x[n x n_in]) in FP32, in row slices of kMlpForwardSlice; work
// holds 2 min(n, kMlpForwardSlice) max_width floats.
constexpr int64_t kMlpForwardSlice = int64_t(1) << 20;
cudaError_t mlp_forward_fp32(const MlpLayout &L, const float *params, const float *x, int64_t n, float *work,
                             float *y, cudaStream_t s);
// Loss partials (npartial doubles, sum / n = MSE) and the packed gradient of
// the MSE of one batch; acts holds mlp_train_floats(L, n) floats.
cudaError_t mlp_loss_grad(const MlpLayout &L, const float *params, const float *x, const float *t, int64_t n,
                          float *acts, float *grad, double *partial, int npartial, cudaStream_t s);
size_t mlp_train_floats(const MlpLayout &L, int64_t n);
// BF16 tensor-core inference (k_mlp_tc.cu): hidden widths equal, a multiple
// of 32 and at most 256, n_in <= 10, scalar output.
bool mlp_bf16_supported(const MlpLayout &L);
size_t mlp_bf16_image_bytes(const MlpLayout &L);
// Rounds the weights into the pre-swizzled bf16 operand image (device).
cudaError_t mlp_bf16_prepare(const MlpLayout &L, const float *params, uint8_t *img, cudaStream_t s);
// y[n] = net(x) with bf16 operands and FP32 accumulation; *err is set to 1
// (and the affected rows to NaN) if a bounded wait of the kernel expires.
cudaError_t mlp_forward_bf16(const MlpLayout &L, const float *params, const uint8_t *img, const float *x, int64_t n,
                             float *y, unsigned int *err, uint32_t cap, cudaStream_t s);
cudaError_t mlp_adam(int64_t count, float *p, const float *g, float *m, float *v, float lr, int step, cudaStream_t s);

}  // namespace gbmc
