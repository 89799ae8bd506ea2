// The pricing surrogate's network: fully connected layers with SiLU
// activations and a scalar linear output (the DNN-layer / simulation-step
// analogy of Sec. III.C), its MSE training by back-propagation (Sec. I.A.3)
// with Adam, all in this file's kernels:
//   gemm_kernel      C = op(A) op(B) (+ bias, + SiLU) in FP32, 64x64 tiles
//   silu_bwd_kernel  dZ = dH * silu'(Z)
//   colsum_kernel    db = column sums of dZ
//   mse_kernel       residual gradient 2 (y - t) / n and loss partials
//   adam_kernel      Adam update of the packed FP32 master parameters
// plus the host runtime behind mc_mlp_* (include/mc.h).  Inference in BF16
// on the tensor cores lives in k_mlp_tc.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mc_kernels.cuh"
#include "mlp.cuh"

namespace gbmc {
namespace {

constexpr int kT = 64, kK = 16;
constexpr int kMaxSlices = 16;  // K slices of a weight-gradient product

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// C[M x N] = op(A)[M x K] * op(B)[K x N]; TA: A stored K x M; TB: B stored N x K.
// Epilogue: v = acc + bias[n]; Z = v (if Z); H = silu(v) or v (if H).
// Split K (grid.z > 1): slice z sums k in [z kchunk, (z + 1) kchunk) and
// writes its partial product at Z + z M ldc (summed by sum_slices_kernel).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                   const float *__restrict__ B, int ldb, const float *__restrict__ bias,
                                                   float *__restrict__ Z, float *__restrict__ H, int ldc, int act,
                                                   int kchunk)
{
    __shared__ float As[kK][kT + 4];
    __shared__ float Bs[kK][kT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * kT, n0 = blockIdx.y * kT;  // row tiles on x: up to 2^31 - 1 blocks
    float acc[4][4] = {};
    const int kb0 = blockIdx.z * kchunk, kend = min(K, kb0 + kchunk);
    if (gridDim.z > 1) {
        Z += static_cast<int64_t>(blockIdx.z) * M * ldc;
        K = kend;
    }
    for (int k0 = kb0; k0 < K; k0 += kK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            int m, k;
            if (TA) { m = e & 63; k = e >> 6; } else { m = e >> 4; k = e & 15; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.0f;
            if (gm < M && gk < K) v = TA ? A[static_cast<int64_t>(gk) * lda + gm] : A[static_cast<int64_t>(gm) * lda + gk];
            As[k][m] = v;
            int n, kb;
            if (TB) { kb = e & 15; n = e >> 4; } else { kb = e >> 6; n = e & 63; }
            const int gn = n0 + n, gkb = k0 + kb;
            float w = 0.0f;
            if (gn < N && gkb < K) w = TB ? B[static_cast<int64_t>(gn) * ldb + gkb] : B[static_cast<int64_t>(gkb) * ldb + gn];
            Bs[kb][n] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const float v = acc[i][j] + (bias ? bias[n] : 0.0f);
            const int64_t o = static_cast<int64_t>(m) * ldc + n;
            if (Z) Z[o] = v;
            if (H) H[o] = act ? silu_f(v) : v;
        }
    }
}

// out[i] = sum_z part[z count + i] (the K slices of a split product, in order).
__global__ void sum_slices_kernel(int64_t count, int slices, const float *part, float *out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < slices; ++z) s += part[static_cast<int64_t>(z) * count + i];
        out[i] = s;
    }
}

__global__ void silu_bwd_kernel(int64_t count, const float *dH, const float *Zv, float *dZ)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dZ[i] = dH[i] * silu_grad_f(Zv[i]);
}

// db[n] = sum_m dZ[m][n]; one block per column group, FP32 with a fixed order.
__global__ void colsum_kernel(int M, int N, const float *dZ, float *db)
{
    const int n = blockIdx.x;
    float s = 0.0f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += dZ[static_cast<int64_t>(m) * N + n];
    s = warp_sum(s);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += ws[w];
        db[n] = t;
    }
}

// dy = 2 (y - t) / n; per-block partial sums of (y - t)^2 in FP64.
__global__ void mse_kernel(int64_t n, const float *y, const float *t, float *dy, double *partial)
{
    double s = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float r = y[i] - t[i];
        dy[i] = 2.0f * r / static_cast<float>(n);
        s += static_cast<double>(r) * r;
    }
    s = warp_sum_d(s);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += ws[w];
        partial[blockIdx.x] = tot;
    }
}

__global__ void adam_kernel(int64_t count, float *p, const float *g, float *m, float *v, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int grid_for(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    return static_cast<int>(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, const float *bias, float *Z,
                 float *H, int ldc, int act, cudaStream_t s)
{
    dim3 grid((M + kT - 1) / kT, (N + kT - 1) / kT);
    gemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, Z, H, ldc, act, K);
    return cudaGetLastError();
}

// C = op(A) op(B) with K cut into `slices` pieces (no bias, no activation):
// partial products into ws [slices][M][N], then one ordered sum into C.
template <bool TA, bool TB>
cudaError_t gemm_split_k(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int slices,
                         float *ws, cudaStream_t s)
{
    const int kchunk = ((K + slices - 1) / slices + kK - 1) / kK * kK;
    slices = (K + kchunk - 1) / kchunk;
    dim3 grid((M + kT - 1) / kT, (N + kT - 1) / kT, slices);
    gemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, nullptr, ws, nullptr, N, 0, kchunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t count = static_cast<int64_t>(M) * N;
    sum_slices_kernel<<<grid_for(count), 256, 0, s>>>(count, slices, ws, C);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------ runtime ----------------------------------
MlpLayout::MlpLayout(int n_in, int width, int hidden)
{
    sizes.push_back(n_in);
    for (int i = 0; i < hidden; ++i) sizes.push_back(width);
    sizes.push_back(1);
    int64_t o = 0;
    for (size_t l = 0; l + 1 < sizes.size(); ++l) {
        w_off.push_back(o);
        o += static_cast<int64_t>(sizes[l]) * sizes[l + 1];
        b_off.push_back(o);
        o += sizes[l + 1];
    }
    count = o;
}

cudaError_t mlp_forward_fp32(const MlpLayout &L, const float *params, const float *x, int64_t n, float *work,
                             float *y, cudaStream_t s)
{
    // work: activations ping-pong, 2 x min(n, 2^20) x max width; rows in slices of 2^20
    int maxw = 0;
    for (int v : L.sizes) maxw = v > maxw ? v : maxw;
    const int nl = static_cast<int>(L.sizes.size()) - 1;
    constexpr int64_t kSlice = kMlpForwardSlice;
    for (int64_t r0 = 0; r0 < n; r0 += kSlice) {
        const int rows = static_cast<int>(n - r0 < kSlice ? n - r0 : kSlice);
        const float *h = x + r0 * L.sizes[0];
        float *buf[2] = {work, work + static_cast<int64_t>(rows) * maxw};
        for (int l = 0; l < nl; ++l) {
            const bool last = l == nl - 1;
            float *out = last ? y + r0 : buf[l & 1];
            cudaError_t e = gemm<false, false>(rows, L.sizes[l + 1], L.sizes[l], h, L.sizes[l], params + L.w_off[l],
                                               L.sizes[l + 1], params + L.b_off[l], nullptr, out, L.sizes[l + 1],
                                               last ? 0 : 1, s);
            if (e != cudaSuccess) return e;
            h = out;
        }
    }
    return cudaSuccess;
}

// Loss and gradient of one batch: acts holds Z_l and H_l for every layer.
cudaError_t mlp_loss_grad(const MlpLayout &L, const float *params, const float *x, const float *t, int64_t n,
                          float *acts, float *grad, double *partial, int npartial, cudaStream_t s)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1;
    // layout of acts: for l = 0..nl-1: Z_l [n x out_l], H_{l+1} [n x out_l]; then dH [n x maxw], dZ [n x maxw]
    std::vector<float *> Zp(nl), Hp(nl);
    float *p = acts;
    int maxw = 0;
    for (int l = 0; l < nl; ++l) {
        Zp[l] = p; p += n * L.sizes[l + 1];
        Hp[l] = p; p += n * L.sizes[l + 1];
        maxw = L.sizes[l + 1] > maxw ? L.sizes[l + 1] : maxw;
    }
    for (int v : L.sizes) maxw = v > maxw ? v : maxw;
    float *dH = p, *dZ = p + n * maxw, *ws = dZ + n * maxw;  // ws: split-K partials of the weight gradients
    cudaError_t e;
    const float *h = x;
    for (int l = 0; l < nl; ++l) {
        e = gemm<false, false>(static_cast<int>(n), L.sizes[l + 1], L.sizes[l], h, L.sizes[l], params + L.w_off[l],
                               L.sizes[l + 1], params + L.b_off[l], Zp[l], Hp[l], L.sizes[l + 1], l < nl - 1 ? 1 : 0, s);
        if (e != cudaSuccess) return e;
        h = Hp[l];
    }
    mse_kernel<<<npartial, 256, 0, s>>>(n, Hp[nl - 1], t, dZ, partial);  // dZ of the linear output layer
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = nl - 1; l >= 0; --l) {
        const int in = L.sizes[l], out = L.sizes[l + 1];
        if (l < nl - 1) {
            silu_bwd_kernel<<<grid_for(n * out), 256, 0, s>>>(n * out, dH, Zp[l], dZ);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        const float *hin = l == 0 ? x : Hp[l - 1];
        // dW = H_in^T dZ   [in x out]: a small output over a long K, so K is split
        const int slices = static_cast<int>(std::min<int64_t>(kMaxSlices, std::max<int64_t>(1, n / 256)));
        e = slices > 1 ? gemm_split_k<true, false>(in, out, static_cast<int>(n), hin, in, dZ, out, grad + L.w_off[l],
                                                   slices, ws, s)
                       : gemm<true, false>(in, out, static_cast<int>(n), hin, in, dZ, out, nullptr, nullptr,
                                           grad + L.w_off[l], out, 0, s);
        if (e != cudaSuccess) return e;
        colsum_kernel<<<out, 256, 0, s>>>(static_cast<int>(n), out, dZ, grad + L.b_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l > 0) {
            // dH_in = dZ W^T   [n x in]
            e = gemm<false, true>(static_cast<int>(n), in, out, dZ, out, params + L.w_off[l], out, nullptr, nullptr, dH,
                                  in, 0, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

size_t mlp_train_floats(const MlpLayout &L, int64_t n)
{
    int maxw = 0;
    size_t f = 0;
    for (size_t l = 0; l + 1 < L.sizes.size(); ++l) {
        f += 2 * static_cast<size_t>(n) * L.sizes[l + 1];
    }
    for (int v : L.sizes) maxw = v > maxw ? v : maxw;
    return f + 2 * static_cast<size_t>(n) * maxw + static_cast<size_t>(kMaxSlices) * maxw * maxw;
}

cudaError_t mlp_adam(int64_t count, float *p, const float *g, float *m, float *v, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, static_cast<float>(step)), c2 = 1.0f - std::pow(b2, static_cast<float>(step));
    adam_kernel<<<grid_for(count), 256, 0, s>>>(count, p, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace gbmc
