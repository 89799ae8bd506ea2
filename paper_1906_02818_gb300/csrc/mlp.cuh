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
// Loss with derivative labels: (1/n) sum [(y - t)^2 + sum_k weight_k m (scale_k
// dy/dx_{dirs_k} - g_k)^2] (m = 1 where g_k is finite) and its gradient, in
// FP32 SIMT products; K <= 4 directions; g [n x K]; acts holds
// mlp_train_floats_d(L, n, K) floats; partial (1 + K) npartial doubles (the
// price part's block sums, then each direction's; divide by n).
constexpr int kMlpMaxDirs = 4;
size_t mlp_train_floats_d(const MlpLayout &L, int64_t n, int K);
cudaError_t mlp_loss_grad_d(const MlpLayout &L, const float *params, const float *x, const float *t, const float *g,
                            int64_t n, int K, const int *dirs, const float *scale, const float *weight, float *acts,
                            float *grad, double *partial, int npartial, cudaStream_t s);
// The same with the width -> width products on the tensor cores (three-pass
// TF32) when mlp_tc_supported(L); acts holds mlp_train_floats_tc(L, n)
// floats; *err is set to 1 if a bounded wait of the tensor-core kernel expires.
bool mlp_tc_supported(const MlpLayout &L);
size_t mlp_train_floats_tc(const MlpLayout &L, int64_t n);
// Derivative-label loss with the width -> width products on the tensor cores
// (three-pass TF32); acts holds mlp_train_floats_d_tc(L, n, K) floats.
size_t mlp_train_floats_d_tc(const MlpLayout &L, int64_t n, int K);
cudaError_t mlp_loss_grad_d_tc(const MlpLayout &L, const float *params, const float *x, const float *t,
                               const float *g, int64_t n, int K, const int *dirs, const float *scale,
                               const float *weight, float *acts, float *grad, double *partial, int npartial,
                               unsigned int *err, uint32_t cap, cudaStream_t s);
cudaError_t mlp_loss_grad_tc(const MlpLayout &L, const float *params, const float *x, const float *t, int64_t n,
                             float *acts, float *grad, double *partial, int npartial, unsigned int *err, uint32_t cap,
                             cudaStream_t s);
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
// Data-parallel building blocks: out[0..count) = n grad, out[count] = sum of
// the loss partials; g = scale src.
cudaError_t mlp_sums_out(int64_t count, const float *grad, double n, const double *partial, int npartial, float *out,
                         cudaStream_t s);
cudaError_t mlp_scale_copy(int64_t count, const float *src, float scale, float *g, cudaStream_t s);

// SiLU and its derivative in FP32 (the training path's activation).
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// Tensor-core training GEMM (k_mlp_tf32.cu): C[M x N] = A[M x K] B[N x K]^T,
// A and B K-major FP32 (row strides lda, ldb, multiples of 4 floats; 16-byte
// aligned bases; any K), three-pass TF32 products with FP32
// accumulation; grid M/128 x N/64 x slices, slice z covering K columns
// [z kchunk, (z + 1) kchunk) (kchunk a multiple of 32).  Epilogues:
constexpr int kTfFwd = 0;   // Z = C + bias, H = silu(Z) ([M x ldc]), Ht = H^T ([N x ldt])
constexpr int kTfBwd = 1;   // dZ = C * silu'(Zin) ([M x ldc]), dZt = dZ^T ([N x ldt])
constexpr int kTfPart = 2;  // P[z][M][N] = C of slice z
struct TfGemmArgs {
    const float *A;
    int64_t lda;
    const float *B;
    int64_t ldb;
    int64_t M;
    int N, K, kchunk;
    int mode;
    const float *bias;
    float *Z, *H, *Ht;
    const float *Zin;
    float *dZ, *dZt;
    float *P;
    int64_t ldc, ldt;
    unsigned int *err;   // set to 1 when a bounded wait expires
    uint32_t cap;        // polls per wait
};
size_t tf32_gemm_smem();
cudaError_t tf32_gemm(const TfGemmArgs &a, int slices, cudaStream_t s);

}  // namespace gbmc
