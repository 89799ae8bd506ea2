// The pricing surrogate's network: fully connected layers with SiLU
// activations and a scalar linear output (the DNN-layer / simulation-step
// analogy of Sec. III.C), its MSE training by back-propagation (Sec. I.A.3)
// with Adam, all in this file's kernels:
//   gemm_kernel      C = op(A) op(B) (+ bias, + SiLU) in FP32, 64x64 tiles, 8x8 per thread
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
constexpr int kGemmThreads = 64;  // threads of gemm_kernel (8 x 8 outputs each)
constexpr int kMaxSlices = 64;    // K slices of a weight-gradient product


// Epilogue of the products: rows m < bias_rows take v = acc + bias[n],
// Z = v (if Z) and H = silu(v) or v (if H); rows at or past bias_rows (the
// tangent rows stacked below a layer's primal rows) take Z = acc only.
__device__ __forceinline__ void store_out(int m, int n, float acc, const float *bias, float *Z, float *H, int ldc,
                                          int act, int bias_rows)
{
    const int64_t o = static_cast<int64_t>(m) * ldc + n;
    if (m < bias_rows) {
        const float v = acc + (bias ? bias[n] : 0.0f);
        if (Z) Z[o] = v;
        if (H) H[o] = act ? silu_f(v) : v;
    } else if (Z) {
        Z[o] = acc;
    }
}

// C[M x N] = op(A)[M x K] * op(B)[K x N]; TA: A stored K x M; TB: B stored N x K.
// Epilogue: store_out.
// Split K (grid.z > 1): slice z sums k in [z kchunk, (z + 1) kchunk) and
// writes its partial product at Z + z M ldc (summed by sum_slices_kernel).
//
// 64 x 64 tiles, 64 threads, each an 8 x 8 block of C: rows
// {4 ty + i} u {32 + 4 ty + i} and columns {4 tx + j} u {32 + 4 tx + j}
// (i, j < 4), so that the 16-byte shared loads of a quarter warp touch
// distinct banks.  Per k a thread reads 8 + 8 values for 64 products, in
// packed FP32x2 FMAs over column pairs (each lane an ordinary FP32 fma, k in
// order): the shared-memory port keeps pace with the FMA pipe, which a
// 4 x 4 block per thread (8 values per 16 products) cannot.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads, 8) gemm8_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                             const float *__restrict__ B, int ldb,
                                                             const float *__restrict__ bias, float *__restrict__ Z,
                                                             float *__restrict__ H, int ldc, int act, int kchunk,
                                                             int bias_rows)
{
    // Rows of 68 floats (272 bytes) keep every 4-float group 16-byte aligned.
    __shared__ __align__(16) float As[kK][kT + 4];
    __shared__ __align__(16) float Bs[kK][kT + 4];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int m0 = blockIdx.x * kT, n0 = blockIdx.y * kT;  // row tiles on x: up to 2^31 - 1 blocks
    // acc2[i][h]: row i of this thread's 8, column pair h (columns 4 tx + 2h,
    // + 1 for h < 2; 32 + 4 tx + 2 (h - 2), + 1 for h >= 2)
    f32x2 acc2[8][4] = {};
    const int kb0 = blockIdx.z * kchunk, kend = min(K, kb0 + kchunk);
    if (gridDim.z > 1) {
        Z += static_cast<int64_t>(blockIdx.z) * M * ldc;
        K = kend;
    }
    for (int k0 = kb0; k0 < K; k0 += kK) {
#pragma unroll
        for (int r = 0; r < (kT * kK) / kGemmThreads; ++r) {
            const int e = tid + kGemmThreads * r;
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
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][32 + ty * 4]);
            const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(&Bs[k][tx * 4]);
            const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(&Bs[k][32 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const f32x2 ai = pack2(av[i], av[i]);
                acc2[i][0] = ffma2(ai, b0.x, acc2[i][0]);
                acc2[i][1] = ffma2(ai, b0.y, acc2[i][1]);
                acc2[i][2] = ffma2(ai, b1.x, acc2[i][2]);
                acc2[i][3] = ffma2(ai, b1.y, acc2[i][3]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? ty * 4 + i : 32 + ty * 4 + (i - 4));
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + (j < 4 ? tx * 4 + j : 32 + tx * 4 + (j - 4));
            if (n >= N) continue;
            const f32x2 pr = acc2[i][j >> 1];
            store_out(m, n, (j & 1) ? hi_of(pr) : lo_of(pr), bias, Z, H, ldc, act, bias_rows);
        }
    }
}

// The 64 x 64 tile with 256 threads of 4 x 4 outputs: more warps for the
// same tile count, used where the 8 x 8 form would leave SMs short of warps
// (a few hundred tiles or fewer).  Same arguments and k order.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm4_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                    const float *__restrict__ B, int ldb, const float *__restrict__ bias,
                                                    float *__restrict__ Z, float *__restrict__ H, int ldc, int act,
                                                    int kchunk, int bias_rows)
{
    __shared__ __align__(16) float As[kK][kT + 4];
    __shared__ __align__(16) float Bs[kK][kT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * kT, n0 = blockIdx.y * kT;
    f32x2 acc2[4][2] = {};
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
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&Bs[k][tx * 4]);
            const f32x2 ai[4] = {pack2(a.x, a.x), pack2(a.y, a.y), pack2(a.z, a.z), pack2(a.w, a.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc2[i][0] = ffma2(ai[i], b.x, acc2[i][0]);
                acc2[i][1] = ffma2(ai[i], b.y, acc2[i][1]);
            }
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
            const f32x2 pr = acc2[i][j >> 1];
            store_out(m, n, (j & 1) ? hi_of(pr) : lo_of(pr), bias, Z, H, ldc, act, bias_rows);
        }
    }
}

// Few inner terms (K <= kSmallK, e.g. the network's input layer): one
// thread per output, k in order.
constexpr int kSmallK = 16;
template <bool TB>
__global__ void smallk_kernel(int M, int N, int K, const float *__restrict__ A, int lda, const float *__restrict__ B,
                              int ldb, const float *__restrict__ bias, float *__restrict__ Z, float *__restrict__ H,
                              int ldc, int act, int bias_rows)
{
    const int64_t total = static_cast<int64_t>(M) * N;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(e / N), n = static_cast<int>(e % N);
        const float *a = A + static_cast<int64_t>(m) * lda;
        float acc = 0.0f;
        for (int k = 0; k < K; ++k) acc = fmaf(a[k], TB ? B[static_cast<int64_t>(n) * ldb + k] : B[static_cast<int64_t>(k) * ldb + n], acc);
        store_out(m, n, acc, bias, Z, H, ldc, act, bias_rows);
    }
}

// One output column (N = 1, e.g. the network's scalar output layer): a warp
// per row, lanes over k, then a fixed-order warp sum.
__global__ void rowvec_kernel(int M, int K, const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
                              const float *__restrict__ bias, float *__restrict__ Z, float *__restrict__ H, int ldc,
                              int act, int bias_rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t m = w0; m < M; m += nw) {
        const float *a = A + m * lda;
        float acc = 0.0f;
        for (int k = lane; k < K; k += 32) acc = fmaf(a[k], B[static_cast<int64_t>(k) * ldb], acc);
        acc = warp_sum(acc);
        if (lane == 0) store_out(static_cast<int>(m), 0, acc, bias, Z, H, ldc, act, bias_rows);
    }
}

// Weight gradients with one small side, partial sums over a chunk of rows:
// part[z][i][c] = sum over rows r of chunk z of X[r][i] Y[r][c], with
// i < I <= kColDotMaxI (X [R x I], Y [R x C], row-major) -- lanes over c --
// or, with I large and C = 1, lanes over i.  FP32, fixed order; the chunks
// are summed by sum_slices_kernel.
constexpr int kColDotMaxI = 8;
template <bool WIDE_X>
__global__ void __launch_bounds__(256) coldot_kernel(int64_t R, int I, int C, const float *__restrict__ X, int ldx,
                                                     const float *__restrict__ Y, int ldy, int64_t rows_per_chunk,
                                                     float *__restrict__ part)
{
    __shared__ float ws[8][kColDotMaxI][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;  // c (or i when WIDE_X)
    const int64_t r0 = blockIdx.y * rows_per_chunk, r1 = min(R, r0 + rows_per_chunk);
    float acc[kColDotMaxI];
#pragma unroll
    for (int i = 0; i < kColDotMaxI; ++i) acc[i] = 0.0f;
    if (WIDE_X) {
        if (col < I)
            for (int64_t r = r0 + w; r < r1; r += 8) acc[0] = fmaf(X[r * ldx + col], Y[r * ldy], acc[0]);
    } else if (col < C) {
        for (int64_t r = r0 + w; r < r1; r += 8) {
            const float y = Y[r * ldy + col];
#pragma unroll
            for (int i = 0; i < kColDotMaxI; ++i)
                if (i < I) acc[i] = fmaf(X[r * ldx + i], y, acc[i]);
        }
    }
    const int ni = WIDE_X ? 1 : I;
    for (int i = 0; i < ni; ++i) ws[w][i][lane] = acc[i];
    __syncthreads();
    if (w == 0) {
        const int64_t slice = WIDE_X ? static_cast<int64_t>(I) : static_cast<int64_t>(I) * C;
        for (int i = 0; i < ni; ++i) {
            float t = 0.0f;
            for (int q = 0; q < 8; ++q) t += ws[q][i][lane];
            if (WIDE_X ? col < I : col < C)
                part[blockIdx.y * slice + (WIDE_X ? col : static_cast<int64_t>(i) * C + col)] = t;
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

// dst[c][r] = src[r][c] for a rows x cols block (32 x 32 shared tiles).
__global__ void transpose_kernel(int64_t rows, int cols, const float *src, int64_t lds, float *dst, int64_t ldd)
{
    __shared__ float tile[32][33];
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = src[r * lds + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[static_cast<int64_t>(c) * ldd + r] = tile[threadIdx.x][i];
    }
}

// out[r] = sum_c src[r][c] (one block per row, FP32 in a fixed order).
__global__ void rowsum_kernel(int cols, const float *src, int64_t ld, float *out)
{
    const float *row = src + static_cast<int64_t>(blockIdx.x) * ld;
    float s = 0.0f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += row[c];
    s = warp_sum(s);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += ws[w];
        out[blockIdx.x] = t;
    }
}

// Skinny products over the batch: for row f of Mt [F x ld] (one block each)
// out[j ldo_j + f] = sum_r Mt[f][r] V[r][j] for j < J (V [n x J], row-major),
// and rsum[f] = sum_r Mt[f][r] if rsum is set.  FP32, fixed order.
constexpr int kRowDotMaxJ = 16;
__global__ void rowdot_kernel(int64_t n, const float *Mt, int64_t ld, const float *V, int J, float *out,
                              int64_t ldo_j, float *rsum)
{
    const int f = blockIdx.x;
    const float *row = Mt + static_cast<int64_t>(f) * ld;
    float acc[kRowDotMaxJ + 1];
#pragma unroll
    for (int j = 0; j <= kRowDotMaxJ; ++j) acc[j] = 0.0f;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const float m = row[r];
#pragma unroll
        for (int j = 0; j < kRowDotMaxJ; ++j)
            if (j < J) acc[j] = fmaf(m, V[r * J + j], acc[j]);
        acc[kRowDotMaxJ] += m;
    }
    __shared__ float ws[kRowDotMaxJ + 1][32];
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j <= kRowDotMaxJ; ++j) {
        if (j >= J && j < kRowDotMaxJ) continue;
        const float v = warp_sum(acc[j]);
        if (lane == 0) ws[j][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < J || (rsum && threadIdx.x == kRowDotMaxJ)) {
        const int j = threadIdx.x;
        float t = 0.0f;
        for (int q = 0; q < nw; ++q) t += ws[j][q];
        if (j < J) out[j * ldo_j + f] = t;
        else rsum[f] = t;
    }
}

// dZ[r][c] = dy[r] w[c] silu'(Z[r][c]) (the output layer's input gradient
// through the last activation) in both layouts: dZ [n x C] and dZt [C x ldt]
// (32 x 32 shared tiles).
__global__ void outer_silu_bwd_kernel(int64_t n, int C, const float *dy, const float *w, const float *Z, float *dZ,
                                      float *dZt, int64_t ldt)
{
    __shared__ float tile[32][33];
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        if (r < n && c < C) {
            const int64_t o = r * C + c;
            const float v = dy[r] * w[c] * silu_grad_f(Z[o]);
            dZ[o] = v;
            tile[i][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (r < n && c < C) dZt[static_cast<int64_t>(c) * ldt + r] = tile[threadIdx.x][i];
    }
}

// out[n][m] = sum_z part[z][m][n] (split-K partials of W^T summed into W).
__global__ void sum_slices_t_kernel(int M, int N, int slices, const float *part, float *out)
{
    const int64_t count = static_cast<int64_t>(M) * N;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(i / N), n = static_cast<int>(i % N);
        float s = 0.0f;
        for (int z = 0; z < slices; ++z) s += part[static_cast<int64_t>(z) * count + i];
        out[static_cast<int64_t>(n) * M + m] = s;
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

// ------------------- derivative labels (input-gradient loss) -------------------
// Rows of a stacked buffer [(K + 1) n x C]: rows 0..n-1 the primal values,
// rows (1 + k) n + i the tangent of direction k for sample i.

constexpr int kMaxDirs = 4;
struct DirSet {
    int K;
    int dir[kMaxDirs];
    float scale[kMaxDirs], weight[kMaxDirs];
};

// Layer 0's tangents: dz = e_{j_k} W_0 = row j_k of W_0 for every sample, and
// dh = silu'(z) dz.  Zs, Hs: [(K + 1) n x C] (primal rows already written).
__global__ void tangent_first_kernel(int64_t n, int C, const float *__restrict__ W0, const DirSet ds,
                                     float *__restrict__ Zs, float *__restrict__ Hs)
{
    const int64_t tot = static_cast<int64_t>(ds.K) * n * C;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(e % C);
        const int64_t ki = e / C, i = ki % n;
        const int k = static_cast<int>(ki / n);
        const float dz = W0[static_cast<int64_t>(ds.dir[k]) * C + c];
        Zs[n * C + e] = dz;
        Hs[n * C + e] = silu_grad_f(Zs[i * C + c]) * dz;
    }
}

// Hidden layers' tangents through the activation: Hs[tangent rows] =
// silu'(z) Zs[tangent rows] with z the sample's primal pre-activation.
__global__ void tangent_act_kernel(int64_t n, int K, int C, const float *__restrict__ Zs, float *__restrict__ Hs)
{
    const int64_t tot = static_cast<int64_t>(K) * n * C;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = (e / C) % n;
        const int c = static_cast<int>(e % C);
        Hs[n * C + e] = silu_grad_f(Zs[i * C + c]) * Zs[n * C + e];
    }
}

// Seeds of the reverse sweep and the loss parts.  Ys: [(K + 1) n] outputs
// (y, then dy/dx_{j_k}); g: [n x K] labels (non-finite: none).  Writes
// Ybar = 2 (y - t) / n and 2 w_k m s_k (s_k dy_k - g_k) / n, and per block the
// FP64 sums of (y - t)^2 and w_k m (s_k dy_k - g_k)^2 at partial[part * nb + block].
__global__ void dloss_seed_kernel(int64_t n, const float *__restrict__ Ys, const float *__restrict__ t,
                                  const float *__restrict__ g, const DirSet ds, float *__restrict__ Ybar,
                                  double *__restrict__ partial)
{
    double acc[1 + kMaxDirs] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const float inv_n = 1.0f / static_cast<float>(n);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float r = Ys[i] - t[i];
        Ybar[i] = 2.0f * r * inv_n;
        acc[0] += static_cast<double>(r) * r;
#pragma unroll
        for (int k = 0; k < kMaxDirs; ++k) {
            if (k >= ds.K) break;
            const float gk = g[i * ds.K + k];
            const bool m = isfinite(gk);
            const float rd = m ? fmaf(ds.scale[k], Ys[(1 + k) * n + i], -gk) : 0.0f;
            Ybar[(1 + k) * n + i] = 2.0f * ds.weight[k] * ds.scale[k] * rd * inv_n;
            acc[1 + k] += static_cast<double>(ds.weight[k]) * rd * rd;
        }
    }
    __shared__ double ws[1 + kMaxDirs][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k <= ds.K; ++k) {
        const double v = warp_sum_d(acc[k]);
        if (lane == 0) ws[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x <= ds.K) {
        double tot = 0.0;
        for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) tot += ws[threadIdx.x][q];
        partial[threadIdx.x * gridDim.x + blockIdx.x] = tot;
    }
}

// Reverse step through h = silu(z), dh_k = silu'(z) dz_k: given the stacked
// input-side adjoints Abar [(K + 1) n x C] and the stacked pre-activations Zs,
//   zbar   = hbar silu'(z) + sum_k dhbar_k silu''(z) dz_k,
//   dzbar_k = dhbar_k silu'(z).
__global__ void dact_bwd_kernel(int64_t n, int K, int C, const float *__restrict__ Abar, const float *__restrict__ Zs,
                                float *__restrict__ Zbar)
{
    const int64_t tot = n * C;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float z = Zs[e];
        const float sg = 1.0f / (1.0f + expf(-z));
        const float d1 = sg * (1.0f + z * (1.0f - sg));
        const float d2 = sg * (1.0f - sg) * (2.0f + z * (1.0f - 2.0f * sg));
        float zb = Abar[e] * d1;
        for (int k = 0; k < K; ++k) {
            const int64_t o = (1 + k) * tot + e;
            zb = fmaf(Abar[o] * d2, Zs[o], zb);
            Zbar[o] = Abar[o] * d1;
        }
        Zbar[e] = zb;
    }
}

// Layer 0's weight gradient from the tangents: row j_k of dW_0 gains the
// column sums of direction k's adjoint rows (dh_0^k = e_{j_k}).
__global__ void dir_rows_kernel(int64_t n, int C, const float *__restrict__ Zbar, const DirSet ds, float *__restrict__ gW0)
{
    const int c = blockIdx.x, k = blockIdx.y;
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += Zbar[((1 + k) * n + i) * C + c];
    s = warp_sum(s);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += ws[w];
        atomicAdd(gW0 + static_cast<int64_t>(ds.dir[k]) * C + c, tot);  // directions may share an input
    }
}

int grid_for(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    return static_cast<int>(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

// Tiled products: the 8 x 8-per-thread kernel once the launch has enough
// tiles to keep every SM's warps busy, else the 4 x 4 one.
constexpr int64_t kGemm8MinOutputs = int64_t(1) << 21;  // outputs x K slices

template <bool TA, bool TB>
void launch_tiled(int M, int N, int K, const float *A, int lda, const float *B, int ldb, const float *bias, float *Z,
                  float *H, int ldc, int act, int kchunk, int slices, int bias_rows, cudaStream_t s)
{
    const dim3 grid((M + kT - 1) / kT, (N + kT - 1) / kT, slices);
    if (static_cast<int64_t>(M) * N * slices >= kGemm8MinOutputs)
        gemm8_kernel<TA, TB><<<grid, kGemmThreads, 0, s>>>(M, N, K, A, lda, B, ldb, bias, Z, H, ldc, act, kchunk,
                                                           bias_rows);
    else
        gemm4_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, Z, H, ldc, act, kchunk, bias_rows);
}

// C = op(A) op(B) with the epilogue of store_out (bias and activation on
// rows m < bias_rows; every row when bias_rows < 0).
template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, const float *bias, float *Z,
                 float *H, int ldc, int act, cudaStream_t s, int bias_rows = -1)
{
    if (bias_rows < 0) bias_rows = M;
    if (!TA && N == 1) {
        rowvec_kernel<<<grid_for(static_cast<int64_t>(M) * 32), 256, 0, s>>>(M, K, A, lda, B, ldb, bias, Z, H, ldc, act,
                                                                             bias_rows);
    } else if (!TA && K <= kSmallK) {
        smallk_kernel<TB><<<grid_for(static_cast<int64_t>(M) * N), 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, Z, H,
                                                                                ldc, act, bias_rows);
    } else {
        launch_tiled<TA, TB>(M, N, K, A, lda, B, ldb, bias, Z, H, ldc, act, K, 1, bias_rows, s);
    }
    return cudaGetLastError();
}

// C = op(A) op(B) with K cut into `slices` pieces (no bias, no activation):
// partial products into ws [slices][M][N], then one ordered sum into C.
// Weight gradients with few input features (M <= kColDotMaxI) or one
// output (N = 1) take the row-chunked dot-product kernel instead of tiles.
template <bool TA, bool TB>
cudaError_t gemm_split_k(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int slices,
                         float *ws, cudaStream_t s)
{
    if (TA && !TB && (M <= kColDotMaxI || N == 1)) {
        const int64_t rows = (K + slices - 1) / slices;
        const int chunks = static_cast<int>((K + rows - 1) / rows);
        if (N == 1)
            coldot_kernel<true><<<dim3((M + 31) / 32, chunks), 256, 0, s>>>(K, M, 1, A, lda, B, ldb, rows, ws);
        else
            coldot_kernel<false><<<dim3((N + 31) / 32, chunks), 256, 0, s>>>(K, M, N, A, lda, B, ldb, rows, ws);
        slices = chunks;
    } else {
        const int kchunk = ((K + slices - 1) / slices + kK - 1) / kK * kK;
        slices = (K + kchunk - 1) / kchunk;
        launch_tiled<TA, TB>(M, N, K, A, lda, B, ldb, nullptr, ws, nullptr, N, 0, kchunk, slices, M, s);
    }
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

// FP32 products for the other path kernels (correlation sensitivities of
// wide baskets), through the same tiled kernels.
cudaError_t gemm_f32_abt(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                         cudaStream_t s)
{
    return gemm<false, true>(M, N, K, A, lda, B, ldb, nullptr, C, nullptr, ldc, 0, s);
}

cudaError_t gemm_f32_atb_slices(int M, int N, int K, const float *A, int lda, const float *B, int ldb, int kchunk,
                                float *part, cudaStream_t s)
{
    if (kchunk <= 0 || kchunk % kK != 0) return cudaErrorInvalidValue;
    const int slices = (K + kchunk - 1) / kchunk;
    launch_tiled<true, false>(M, N, K, A, lda, B, ldb, nullptr, part, nullptr, N, 0, kchunk, slices, M, s);
    return cudaGetLastError();
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

size_t mlp_train_floats_d(const MlpLayout &L, int64_t n, int K)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1;
    int maxw = 0;
    size_t f = 0;
    for (int l = 0; l < nl; ++l) f += 2 * static_cast<size_t>(K + 1) * n * L.sizes[l + 1];
    for (int v : L.sizes) maxw = v > maxw ? v : maxw;
    return f + 2 * static_cast<size_t>(K + 1) * n * maxw + static_cast<size_t>(kMaxSlices) * maxw * maxw;
}

// Loss with derivative labels and its gradient: a forward sweep of the
// primal rows and, stacked below them, one tangent per direction
// (dz = dh W, next dh = silu'(z) dz); a reverse sweep through both
// (W-bar = h^T z-bar + sum_k dh_k^T dz_k-bar, h-bar = z-bar W^T,
// dh_k-bar = dz_k-bar W^T, previous z-bar = h-bar silu'(z)
// + sum_k dh_k-bar silu''(z) dz_k, previous dz_k-bar = dh_k-bar silu'(z)).
// acts: mlp_train_floats_d floats; partial: (1 + K) npartial doubles.
cudaError_t mlp_loss_grad_d(const MlpLayout &L, const float *params, const float *x, const float *t, const float *g,
                            int64_t n, int K, const int *dirs, const float *scale, const float *weight, float *acts,
                            float *grad, double *partial, int npartial, cudaStream_t s)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1;
    const int64_t R = (K + 1) * n;  // stacked rows
    DirSet ds{};
    ds.K = K;
    for (int k = 0; k < K; ++k) {
        ds.dir[k] = dirs[k];
        ds.scale[k] = scale[k];
        ds.weight[k] = weight[k];
    }
    std::vector<float *> Zs(nl), Hs(nl);  // Zs[l]: pre-activations of layer l; Hs[l]: its outputs (stacked)
    float *p = acts;
    int maxw = 0;
    for (int l = 0; l < nl; ++l) {
        Zs[l] = p; p += R * L.sizes[l + 1];
        Hs[l] = p; p += R * L.sizes[l + 1];
    }
    for (int v : L.sizes) maxw = v > maxw ? v : maxw;
    float *Abar = p, *Zbar = p + R * maxw, *ws = Zbar + R * maxw;
    cudaError_t e;
    // forward
    for (int l = 0; l < nl; ++l) {
        const int in = L.sizes[l], out = L.sizes[l + 1];
        const bool last = l == nl - 1;
        const float *hin = l == 0 ? x : Hs[l - 1];
        // layer 0: the primal rows (tangents by tangent_first_kernel); later
        // layers: primal and tangent rows in one product, bias and activation
        // on the primal rows only (the tangents' H by tangent_act_kernel)
        const int64_t rows = (l == 0 || K == 0) ? n : R;
        e = gemm<false, false>(static_cast<int>(rows), out, in, hin, in, params + L.w_off[l], out, params + L.b_off[l],
                               Zs[l], last ? nullptr : Hs[l], out, last ? 0 : 1, s, static_cast<int>(n));
        if (e != cudaSuccess) return e;
        if (K == 0) continue;
        if (l == 0) {
            tangent_first_kernel<<<grid_for(K * n * out), 256, 0, s>>>(n, out, params + L.w_off[0], ds, Zs[0], Hs[0]);
        } else if (!last) {
            tangent_act_kernel<<<grid_for(K * n * out), 256, 0, s>>>(n, K, out, Zs[l], Hs[l]);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // seeds: the output layer's stacked pre-activations are (y, dy/dx_{j_k})
    dloss_seed_kernel<<<npartial, 256, 0, s>>>(n, Zs[nl - 1], t, g, ds, Zbar, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = nl - 1; l >= 0; --l) {
        const int in = L.sizes[l], out = L.sizes[l + 1];
        const int64_t rows = l == 0 ? n : R;  // layer 0's tangent inputs are unit vectors (dir_rows_kernel)
        const float *hin = l == 0 ? x : Hs[l - 1];
        const int slices = static_cast<int>(std::min<int64_t>(kMaxSlices, std::max<int64_t>(1, rows / 256)));
        e = slices > 1 ? gemm_split_k<true, false>(in, out, static_cast<int>(rows), hin, in, Zbar, out,
                                                   grad + L.w_off[l], slices, ws, s)
                       : gemm<true, false>(in, out, static_cast<int>(rows), hin, in, Zbar, out, nullptr, nullptr,
                                           grad + L.w_off[l], out, 0, s);
        if (e != cudaSuccess) return e;
        if (l == 0 && K > 0) {
            dir_rows_kernel<<<dim3(out, K), 256, 0, s>>>(n, out, Zbar, ds, grad + L.w_off[0]);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        colsum_kernel<<<out, 256, 0, s>>>(static_cast<int>(n), out, Zbar, grad + L.b_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l > 0) {
            e = gemm<false, true>(static_cast<int>(R), in, out, Zbar, out, params + L.w_off[l], out, nullptr, nullptr,
                                  Abar, in, 0, s);
            if (e != cudaSuccess) return e;
            dact_bwd_kernel<<<grid_for(n * in), 256, 0, s>>>(n, K, in, Abar, Zs[l - 1], Zbar);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Tensor-core training (k_mlp_tf32.cu) covers the width -> width layers:
// sizes n_in, W x hidden, 1 with hidden >= 2 and W a multiple of 64.
bool mlp_tc_supported(const MlpLayout &L)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1;
    if (nl < 3 || L.sizes[nl] != 1) return false;
    const int W = L.sizes[1];
    if (W % 64 != 0) return false;
    for (int l = 1; l < nl; ++l)
        if (L.sizes[l] != W) return false;
    return true;
}

namespace {
constexpr int kTcMaxSlices = 32;
int64_t round4(int64_t n) { return (n + 3) / 4 * 4; }
}  // namespace

size_t mlp_train_floats_tc(const MlpLayout &L, int64_t n)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1, W = L.sizes[1];
    const size_t nt = static_cast<size_t>(round4(n));
    size_t f = 0;
    for (int l = 0; l < nl; ++l) f += 2 * static_cast<size_t>(n) * L.sizes[l + 1];  // Z, H
    f += static_cast<size_t>(nl - 1) * W * nt;                                      // H^T of the hidden layers
    f += 3 * static_cast<size_t>(n) * W + 2 * static_cast<size_t>(W) * nt;           // dH, dZ[2], dZt[2]
    f += static_cast<size_t>(nl - 2) * W * W;                                        // W_l^T
    const int in0 = L.sizes[0];
    f += static_cast<size_t>(std::max(kTcMaxSlices, kMaxSlices)) * std::max(W, in0) * W;  // split-K partials
    return f + 64;  // 16-byte alignment of the pieces
}

// As mlp_loss_grad, with the width -> width layers' forward, input-gradient
// and weight-gradient products on the tensor cores (three-pass TF32, FP32
// accumulation); the input layer, the scalar output layer, the loss and the
// element-wise steps as in mlp_loss_grad.
cudaError_t mlp_loss_grad_tc(const MlpLayout &L, const float *params, const float *x, const float *t, int64_t n,
                             float *acts, float *grad, double *partial, int npartial, unsigned int *err, uint32_t cap,
                             cudaStream_t s)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1, W = L.sizes[1], n_in = L.sizes[0];
    const int64_t nt = round4(n);
    float *p = acts;
    auto take = [&](size_t count) {
        float *q = p;
        p += (count + 3) / 4 * 4;
        return q;
    };
    std::vector<float *> Zp(nl), Hp(nl), Ht(nl - 1), WT(nl - 1, nullptr);
    for (int l = 0; l < nl; ++l) {
        Zp[l] = take(static_cast<size_t>(n) * L.sizes[l + 1]);
        Hp[l] = take(static_cast<size_t>(n) * L.sizes[l + 1]);
    }
    for (int l = 0; l < nl - 1; ++l) Ht[l] = take(static_cast<size_t>(W) * nt);
    float *dH = take(static_cast<size_t>(n) * W);
    float *dZ[2] = {take(static_cast<size_t>(n) * W), take(static_cast<size_t>(n) * W)};
    float *dZt[2] = {take(static_cast<size_t>(W) * nt), take(static_cast<size_t>(W) * nt)};
    for (int l = 1; l < nl - 1; ++l) WT[l] = take(static_cast<size_t>(W) * W);
    float *ws = p;
    cudaError_t e;
    const dim3 tb(32, 8);
    auto transpose = [&](int64_t rows, int cols, const float *src, int64_t lds, float *dst, int64_t ldd) {
        const dim3 g(static_cast<unsigned>((rows + 31) / 32), static_cast<unsigned>((cols + 31) / 32));
        transpose_kernel<<<g, tb, 0, s>>>(rows, cols, src, lds, dst, ldd);
        return cudaGetLastError();
    };
    TfGemmArgs base{};
    base.err = err;
    base.cap = cap;
    // W_l^T (out x in, K-major over in) of the width -> width layers
    for (int l = 1; l < nl - 1; ++l)
        if ((e = transpose(W, W, params + L.w_off[l], W, WT[l], W)) != cudaSuccess) return e;
    // forward
    e = gemm<false, false>(static_cast<int>(n), W, n_in, x, n_in, params + L.w_off[0], W, params + L.b_off[0], Zp[0],
                           Hp[0], W, 1, s);
    if (e != cudaSuccess) return e;
    if ((e = transpose(n, W, Hp[0], W, Ht[0], nt)) != cudaSuccess) return e;
    for (int l = 1; l < nl - 1; ++l) {
        TfGemmArgs a = base;
        a.A = Hp[l - 1]; a.lda = W;
        a.B = WT[l]; a.ldb = W;
        a.M = n; a.N = W; a.K = W; a.kchunk = W;
        a.mode = kTfFwd;
        a.bias = params + L.b_off[l];
        a.Z = Zp[l]; a.H = Hp[l]; a.Ht = Ht[l];
        a.ldc = W; a.ldt = nt;
        if ((e = tf32_gemm(a, 1, s)) != cudaSuccess) return e;
    }
    const int lo = nl - 1;  // scalar output layer
    e = gemm<false, false>(static_cast<int>(n), 1, W, Hp[lo - 1], W, params + L.w_off[lo], 1, params + L.b_off[lo],
                           Zp[lo], Hp[lo], 1, 0, s);
    if (e != cudaSuccess) return e;
    float *dy = dZ[1];
    mse_kernel<<<npartial, 256, 0, s>>>(n, Hp[lo], t, dy, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // output layer: dW = H^T dy (from H^T), db = sum dy, dZ = (dy w^T) silu'(Z) in both layouts
    rowdot_kernel<<<W, 256, 0, s>>>(n, Ht[lo - 1], nt, dy, 1, grad + L.w_off[lo], 0, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    colsum_kernel<<<1, 256, 0, s>>>(static_cast<int>(n), 1, dy, grad + L.b_off[lo]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        const dim3 g(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((W + 31) / 32));
        outer_silu_bwd_kernel<<<g, tb, 0, s>>>(n, W, dy, params + L.w_off[lo], Zp[lo - 1], dZ[0], dZt[0], nt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // width -> width layers, l = nl - 2 .. 1: dZ[cur] / dZt[cur] hold dZ_l
    int cur = 0;
    const int slices0 = static_cast<int>(std::min<int64_t>(kTcMaxSlices, std::max<int64_t>(1, (n + 255) / 256)));
    const int kchunk = static_cast<int>(((n + slices0 - 1) / slices0 + 31) / 32 * 32);
    const int slices = static_cast<int>((n + kchunk - 1) / kchunk);
    for (int l = nl - 2; l >= 1; --l) {
        // dW_l^T [out x in] = dZ_l^T H_{l-1}: split-K partials, summed into W's layout
        TfGemmArgs a = base;
        a.A = dZt[cur]; a.lda = nt;
        a.B = Ht[l - 1]; a.ldb = nt;
        a.M = W; a.N = W; a.K = static_cast<int>(n); a.kchunk = kchunk;
        a.mode = kTfPart;
        a.P = ws;
        if ((e = tf32_gemm(a, slices, s)) != cudaSuccess) return e;
        sum_slices_t_kernel<<<grid_for(static_cast<int64_t>(W) * W), 256, 0, s>>>(W, W, slices, ws, grad + L.w_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        rowsum_kernel<<<W, 256, 0, s>>>(static_cast<int>(n), dZt[cur], nt, grad + L.b_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // dZ_{l-1} = (dZ_l W_l^T) silu'(Z_{l-1}): B = W_l [in x out], K-major over out
        TfGemmArgs b = base;
        b.A = dZ[cur]; b.lda = W;
        b.B = params + L.w_off[l]; b.ldb = W;
        b.M = n; b.N = W; b.K = W; b.kchunk = W;
        b.mode = kTfBwd;
        b.Zin = Zp[l - 1];
        b.dZ = dZ[cur ^ 1]; b.dZt = dZt[cur ^ 1];
        b.ldc = W; b.ldt = nt;
        if ((e = tf32_gemm(b, 1, s)) != cudaSuccess) return e;
        cur ^= 1;
    }
    // input layer: dW_0[i][f] = sum_r dZ_0^T[f][r] x[r][i], db_0 = row sums of dZ_0^T
    if (n_in <= kRowDotMaxJ) {
        rowdot_kernel<<<W, 256, 0, s>>>(n, dZt[cur], nt, x, n_in, grad + L.w_off[0], W, grad + L.b_off[0]);
        return cudaGetLastError();
    }
    const int sl0 = static_cast<int>(std::min<int64_t>(kMaxSlices, std::max<int64_t>(1, n / 256)));
    e = sl0 > 1 ? gemm_split_k<true, false>(n_in, W, static_cast<int>(n), x, n_in, dZ[cur], W, grad + L.w_off[0], sl0,
                                             ws, s)
                : gemm<true, false>(n_in, W, static_cast<int>(n), x, n_in, dZ[cur], W, nullptr, nullptr,
                                    grad + L.w_off[0], W, 0, s);
    if (e != cudaSuccess) return e;
    rowsum_kernel<<<W, 256, 0, s>>>(static_cast<int>(n), dZt[cur], nt, grad + L.b_off[0]);
    return cudaGetLastError();
}

namespace {
// Rows r < n of a layer's stacked pre-activations: Z += b, H = silu(Z).
__global__ void bias_act_rows_kernel(int64_t n, int C, const float *__restrict__ b, float *__restrict__ Z,
                                     float *__restrict__ H)
{
    const int64_t tot = n * C;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float z = Z[e] + b[e % C];
        Z[e] = z;
        H[e] = silu_f(z);
    }
}
}  // namespace

size_t mlp_train_floats_d_tc(const MlpLayout &L, int64_t n, int K)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1, W = L.sizes[1];
    const int64_t R = (K + 1) * n, Rt = round4(R);
    size_t f = 0;
    for (int l = 0; l < nl; ++l) f += 2 * static_cast<size_t>(round4(R * L.sizes[l + 1]));  // Z, H (stacked)
    f += 2 * static_cast<size_t>(Rt) * W;                                                   // Abar, Zbar
    f += 2 * static_cast<size_t>(W) * Rt;                                                   // H^T, Zbar^T
    f += static_cast<size_t>(nl - 2) * W * W;                                               // W_l^T
    f += static_cast<size_t>(std::max(kTcMaxSlices, kMaxSlices)) * W * W;                   // split-K partials
    return f + 64;
}

// As mlp_loss_grad_d, with the width -> width layers' three products (the
// stacked forward rows, the input gradient and the weight gradient) on the
// tensor cores in three-pass TF32 (plain row-major outputs, then the same
// element-wise steps as the SIMT path); the input layer, the scalar output
// layer and the element-wise steps unchanged.
cudaError_t mlp_loss_grad_d_tc(const MlpLayout &L, const float *params, const float *x, const float *t,
                               const float *g, int64_t n, int K, const int *dirs, const float *scale,
                               const float *weight, float *acts, float *grad, double *partial, int npartial,
                               unsigned int *err, uint32_t cap, cudaStream_t s)
{
    const int nl = static_cast<int>(L.sizes.size()) - 1, W = L.sizes[1];
    const int64_t R = (K + 1) * n, Rt = round4(R);
    DirSet ds{};
    ds.K = K;
    for (int k = 0; k < K; ++k) {
        ds.dir[k] = dirs[k];
        ds.scale[k] = scale[k];
        ds.weight[k] = weight[k];
    }
    float *p = acts;
    auto take = [&](size_t count) {
        float *q = p;
        p += (count + 3) / 4 * 4;
        return q;
    };
    std::vector<float *> Zs(nl), Hs(nl), WT(nl - 1, nullptr);
    for (int l = 0; l < nl; ++l) {
        Zs[l] = take(static_cast<size_t>(R) * L.sizes[l + 1]);
        Hs[l] = take(static_cast<size_t>(R) * L.sizes[l + 1]);
    }
    float *Abar = take(static_cast<size_t>(Rt) * W), *Zbar = take(static_cast<size_t>(Rt) * W);
    float *Ht = take(static_cast<size_t>(W) * Rt), *Zt = take(static_cast<size_t>(W) * Rt);
    for (int l = 1; l < nl - 1; ++l) WT[l] = take(static_cast<size_t>(W) * W);
    float *ws = p;
    cudaError_t e;
    const dim3 tb(32, 8);
    auto transpose = [&](int64_t rows, int cols, const float *src, int64_t lds, float *dst, int64_t ldd) {
        const dim3 gt(static_cast<unsigned>((rows + 31) / 32), static_cast<unsigned>((cols + 31) / 32));
        transpose_kernel<<<gt, tb, 0, s>>>(rows, cols, src, lds, dst, ldd);
        return cudaGetLastError();
    };
    TfGemmArgs base{};
    base.err = err;
    base.cap = cap;
    base.mode = kTfPart;
    // C [M x N] = A [M x Kd] B [N x Kd]^T into P (row-major, ld N); split K when slices > 1
    auto product = [&](const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int N, int Kd, int slices,
                       float *P) {
        TfGemmArgs a = base;
        a.A = A; a.lda = lda;
        a.B = B; a.ldb = ldb;
        a.M = M; a.N = N; a.K = Kd;
        a.kchunk = slices > 1 ? static_cast<int>(((Kd + slices - 1) / slices + 31) / 32 * 32) : Kd;
        a.P = P;
        const int sl = (Kd + a.kchunk - 1) / a.kchunk;
        cudaError_t r = tf32_gemm(a, sl, s);
        return std::make_pair(r, sl);
    };
    for (int l = 1; l < nl - 1; ++l)
        if ((e = transpose(W, W, params + L.w_off[l], W, WT[l], W)) != cudaSuccess) return e;
    // forward
    for (int l = 0; l < nl; ++l) {
        const int in = L.sizes[l], out = L.sizes[l + 1];
        const bool last = l == nl - 1;
        if (l == 0 || last) {
            const int64_t rows = (l == 0 || K == 0) ? n : R;
            e = gemm<false, false>(static_cast<int>(rows), out, in, l == 0 ? x : Hs[l - 1], in, params + L.w_off[l], out,
                                   params + L.b_off[l], Zs[l], last ? nullptr : Hs[l], out, last ? 0 : 1, s,
                                   static_cast<int>(n));
            if (e != cudaSuccess) return e;
            if (l == 0 && K > 0)
                tangent_first_kernel<<<grid_for(K * n * out), 256, 0, s>>>(n, out, params + L.w_off[0], ds, Zs[0], Hs[0]);
        } else {
            const auto r = product(Hs[l - 1], W, WT[l], W, R, W, W, 1, Zs[l]);
            if ((e = r.first) != cudaSuccess) return e;
            bias_act_rows_kernel<<<grid_for(n * W), 256, 0, s>>>(n, W, params + L.b_off[l], Zs[l], Hs[l]);
            if (K > 0) tangent_act_kernel<<<grid_for(K * n * W), 256, 0, s>>>(n, K, W, Zs[l], Hs[l]);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    dloss_seed_kernel<<<npartial, 256, 0, s>>>(n, Zs[nl - 1], t, g, ds, Zbar, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = nl - 1; l >= 0; --l) {
        const int in = L.sizes[l], out = L.sizes[l + 1];
        const int64_t rows = l == 0 ? n : R;
        const float *hin = l == 0 ? x : Hs[l - 1];
        if (l == 0 || l == nl - 1) {
            const int slices = static_cast<int>(std::min<int64_t>(kMaxSlices, std::max<int64_t>(1, rows / 256)));
            e = slices > 1 ? gemm_split_k<true, false>(in, out, static_cast<int>(rows), hin, in, Zbar, out,
                                                       grad + L.w_off[l], slices, ws, s)
                           : gemm<true, false>(in, out, static_cast<int>(rows), hin, in, Zbar, out, nullptr, nullptr,
                                               grad + L.w_off[l], out, 0, s);
            if (e != cudaSuccess) return e;
        } else {
            // dW_l^T [out x in] = Zbar^T H_{l-1}: both transposed to K-major over the stacked rows
            if ((e = transpose(R, W, Zbar, W, Zt, Rt)) != cudaSuccess) return e;
            if ((e = transpose(R, W, hin, W, Ht, Rt)) != cudaSuccess) return e;
            const int slices0 = static_cast<int>(std::min<int64_t>(kTcMaxSlices, std::max<int64_t>(1, (R + 255) / 256)));
            const auto r = product(Zt, Rt, Ht, Rt, W, W, static_cast<int>(R), slices0, ws);
            if ((e = r.first) != cudaSuccess) return e;
            sum_slices_t_kernel<<<grid_for(static_cast<int64_t>(W) * W), 256, 0, s>>>(W, W, r.second, ws,
                                                                                     grad + L.w_off[l]);
        }
        if (l == 0 && K > 0) dir_rows_kernel<<<dim3(out, K), 256, 0, s>>>(n, out, Zbar, ds, grad + L.w_off[0]);
        colsum_kernel<<<out, 256, 0, s>>>(static_cast<int>(n), out, Zbar, grad + L.b_off[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l > 0) {
            if (l == nl - 1) {
                e = gemm<false, true>(static_cast<int>(R), in, out, Zbar, out, params + L.w_off[l], out, nullptr,
                                      nullptr, Abar, in, 0, s);
            } else {
                // Abar [R x in] = Zbar W_l^T: B = W_l [in x out], K-major over out
                e = product(Zbar, W, params + L.w_off[l], W, R, W, W, 1, Abar).first;
            }
            if (e != cudaSuccess) return e;
            dact_bwd_kernel<<<grid_for(n * in), 256, 0, s>>>(n, K, in, Abar, Zs[l - 1], Zbar);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
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

// out[i] = n grad[i] for i < count (the gradient of the batch's summed loss);
// out[count] = the sum of the loss partials, added by one block in FP64.
__global__ void sums_out_kernel(int64_t count, const float *__restrict__ grad, double n,
                                const double *__restrict__ partial, int npartial, float *__restrict__ out)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = static_cast<float>(n * grad[i]);
    if (blockIdx.x == 0) {
        __shared__ double s_red[8];
        double v = 0.0;
        for (int i = threadIdx.x; i < npartial; i += blockDim.x) v += partial[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += s_red[w];
            out[count] = static_cast<float>(tot);
        }
    }
}

__global__ void scale_copy_kernel(int64_t count, const float *__restrict__ src, float scale, float *__restrict__ g)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        g[i] = scale * src[i];
}

cudaError_t mlp_sums_out(int64_t count, const float *grad, double n, const double *partial, int npartial, float *out,
                         cudaStream_t s)
{
    sums_out_kernel<<<grid_for(count), 256, 0, s>>>(count, grad, n, partial, npartial, out);
    return cudaGetLastError();
}

cudaError_t mlp_scale_copy(int64_t count, const float *src, float scale, float *g, cudaStream_t s)
{
    scale_copy_kernel<<<grid_for(count), 256, 0, s>>>(count, src, scale, g);
    return cudaGetLastError();
}

cudaError_t mlp_adam(int64_t count, float *p, const float *g, float *m, float *v, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, static_cast<float>(step)), c2 = 1.0f - std::pow(b2, static_cast<float>(step));
    adam_kernel<<<grid_for(count), 256, 0, s>>>(count, p, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace gbmc
