// FP64 linear algebra of the set-up phase: the Cholesky factor of the asset
// correlation (Sec. II.A.2 needs a factor sigma with sigma sigma^T equal to
// the covariance; Sec. II.A.3 uses the same factorisation for the Grammian)
// and its scaled FP32 copy for the FP32 contraction.
#include "mc_kernels.cuh"

namespace gbmc {

namespace {


// 1/sqrt(p) for p > 0: an FP32 estimate refined by two Newton steps
// r <- r (3/2 - p r^2 / 2) in FP64 (quadratic convergence: 2^-23 -> 2^-46 ->
// a few ulp); outside FP32's range, FP64 square root and division.  FP64
// division and square root are long serial chains on this part, and the
// factorisation's column loop is serial in them.
__device__ __forceinline__ double rsqrt_refined(double p)
{
    if (!(p > 1e-30 && p < 1e30)) return 1.0 / sqrt(p);
    double r = static_cast<double>(rsqrtf(static_cast<float>(p)));
    r = r * fma(-0.5 * p, r * r, 1.5);
    r = r * fma(-0.5 * p, r * r, 1.5);
    return r;
}

// A pivot at or below kPivotTol A_kk is taken as zero: the matrix is
// rejected as not positive definite.  4 d eps (eps = 2^-52) is a few times the
// rounding a pivot collects over its d updates, so a semi-definite
// (rank-deficient) matrix is rejected whatever that rounding gives, while a
// positive definite one passes unless its conditional variance falls below
// ~1e-13 of its variance (a factor that small, 3e-7, is below FP32 paths'
// resolution anyway).
__device__ __forceinline__ bool pivot_ok(double p, double akk, int d)
{
    return p > 4.0 * d * 2.220446049250313e-16 * akk;
}

// Right-looking Cholesky for d <= 64 in one CTA, W in shared memory: each
// column is scaled by its pivot's reciprocal square root (rsqrt_refined).
// FP64 issue is the scarce resource here (a warp's FP64 instruction holds
// its SM quarter for tens of cycles), so the trailing update of column k
// walks the lower triangle of the (d-k-1)^2 block densely, through a table
// of (row, column) offsets enumerated row by row: every lane of every issued
// FMA does work, and no index needs a division.  Entry 0 of the walk is the
// next pivot, which thread 0 therefore updates itself: it forms the next
// pivot's reciprocal square root without waiting, and each column costs two
// block barriers.
constexpr int kCholSmallD = 64;
constexpr int kCholSmallBlock = 256;
constexpr int kCholTri = (kCholSmallD - 1) * kCholSmallD / 2;  // entries of the largest trailing triangle

__global__ void __launch_bounds__(kCholSmallBlock) cholesky_small_kernel(int d, const double *A, double *L, int *status)
{
    __shared__ double W[kCholSmallD][kCholSmallD + 1];
    __shared__ uint16_t tri[kCholTri];  // (ii << 6) | jj, jj <= ii, row by row
    __shared__ double s_inv;
    __shared__ int s_fail;
    const int t = threadIdx.x;
    for (int idx = t; idx < d * d; idx += blockDim.x) W[idx / d][idx % d] = A[idx];
    for (int ii = t; ii < kCholSmallD - 1; ii += blockDim.x)
        for (int jj = 0; jj <= ii; ++jj) tri[ii * (ii + 1) / 2 + jj] = static_cast<uint16_t>((ii << 6) | jj);
    if (t == 0) {
        s_fail = 0;
        const double p = d > 0 ? A[0] : 1.0;
        if (!pivot_ok(p, p, d)) {
            s_fail = 1;
        } else {
            const double r = rsqrt_refined(p);
            s_inv = r;
        }
    }
    __syncthreads();
    if (t == 0 && !s_fail && d > 0) W[0][0] = W[0][0] * s_inv;  // p r with p = W[0][0]
    for (int k = 0; k < d; ++k) {
        // s_inv holds 1/sqrt of the pivot W[k][k] (thread 0 wrote both)
        __syncthreads();
        if (s_fail) break;
        const double inv = s_inv;
        for (int i = k + 1 + t; i < d; i += blockDim.x) W[i][k] *= inv;
        __syncthreads();
        const int m = d - k - 1, n = m * (m + 1) / 2;
        for (int e = t; e < n; e += blockDim.x) {
            const int code = tri[e], i = k + 1 + (code >> 6), j = k + 1 + (code & 63);
            W[i][j] -= W[i][k] * W[j][k];
        }
        // entry 0 is (k + 1, k + 1), updated above by this same thread
        if (t == 0 && k + 1 < d) {
            const double p = W[k + 1][k + 1];
            if (!pivot_ok(p, A[(k + 1) * d + (k + 1)], d)) {
                s_fail = 1;
            } else {
                const double r = rsqrt_refined(p);
                W[k + 1][k + 1] = p * r;
                s_inv = r;
            }
        }
    }
    __syncthreads();
    if (!s_fail)
        for (int idx = t; idx < d * d; idx += blockDim.x) {
            const int i = idx / d, j = idx % d;
            L[idx] = j > i ? 0.0 : W[i][j];
        }
    if (t == 0) *status = s_fail;
}

// Blocked right-looking Cholesky for d > 64, spread over the SMs (FP64 issue
// on this part is a few FMAs per clock per SM, so one CTA is slow): for each
// 32-column block K, (1) one CTA factors the diagonal block in shared memory,
// (2) one thread per row below it solves the panel row against it, (3) one
// CTA per 32 x 32 block of the trailing lower triangle subtracts the panel
// product.  Pivots are checked against the original diagonal as above.
constexpr int kCholNb = 32;

__global__ void chol_copy_kernel(int64_t n, const double *__restrict__ A, double *__restrict__ W, int *status)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        W[i] = A[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// (1) the diagonal block W[k0 .. k0 + nb)^2, in place (lower part)
__global__ void __launch_bounds__(256) chol_diag_kernel(int d, int k0, int nb, const double *__restrict__ A,
                                                        double *__restrict__ W, int *status)
{
    __shared__ double T[kCholNb][kCholNb + 1];
    __shared__ double s_inv;
    __shared__ int s_fail;
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) T[e / nb][e % nb] = W[static_cast<int64_t>(k0 + e / nb) * d + k0 + e % nb];
    if (t == 0) s_fail = 0;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        if (t == 0) {
            const double p = T[k][k];
            const int64_t g = static_cast<int64_t>(k0 + k) * d + (k0 + k);
            if (!pivot_ok(p, A[g], d)) {
                s_fail = 1;
            } else {
                const double r = rsqrt_refined(p);
                T[k][k] = p * r;
                s_inv = r;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double inv = s_inv;
        for (int i = k + 1 + t; i < nb; i += blockDim.x) T[i][k] *= inv;
        __syncthreads();
        const int m = nb - k - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) T[i][j] -= T[i][k] * T[j][k];
        }
        __syncthreads();
    }
    if (s_fail) {
        if (t == 0) *status = 1;
        return;
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        if (j <= i) W[static_cast<int64_t>(k0 + i) * d + k0 + j] = T[i][j];
    }
}

// (2) rows i >= k0 + nb of the panel: L_ij = (W_ij - sum_{c < j} L_ic L_jc) / L_jj, j in the block
__global__ void chol_panel_kernel(int d, int k0, int nb, double *__restrict__ W)
{
    const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double *Ri = W + static_cast<int64_t>(i) * d + k0;
    for (int j = 0; j < nb; ++j) {
        const double *Rj = W + static_cast<int64_t>(k0 + j) * d + k0;
        double s = Ri[j];
        for (int c = 0; c < j; ++c) s = fma(-Ri[c], Rj[c], s);
        Ri[j] = s / Rj[j];
    }
}

// (3) the trailing lower triangle, one CTA per 32 x 32 block (bi >= bj) of
// rows / columns from k0 + nb: W_ij -= sum_c L_ic L_jc over the panel columns
__global__ void __launch_bounds__(256) chol_update_kernel(int d, int k0, int nb, double *__restrict__ W)
{
    __shared__ double Pi[kCholNb][kCholNb + 1], Pj[kCholNb][kCholNb + 1];
    // blockIdx.x enumerates the lower-triangle blocks row by row
    int bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= static_cast<int>(blockIdx.x)) ++bi;
    const int bj = static_cast<int>(blockIdx.x) - bi * (bi + 1) / 2;
    const int r0 = k0 + nb + bi * kCholNb, c0 = k0 + nb + bj * kCholNb;
    const int t = threadIdx.x;
    for (int e = t; e < kCholNb * kCholNb; e += blockDim.x) {
        const int r = e / kCholNb, c = e % kCholNb;
        Pi[r][c] = (r0 + r < d && c < nb) ? W[static_cast<int64_t>(r0 + r) * d + k0 + c] : 0.0;
        Pj[r][c] = (c0 + r < d && c < nb) ? W[static_cast<int64_t>(c0 + r) * d + k0 + c] : 0.0;
    }
    __syncthreads();
    for (int e = t; e < kCholNb * kCholNb; e += blockDim.x) {
        const int r = e / kCholNb, c = e % kCholNb;
        const int i = r0 + r, j = c0 + c;
        if (i < d && j <= i) {
            double s = 0.0;
            for (int q = 0; q < nb; ++q) s = fma(Pi[r][q], Pj[c][q], s);
            W[static_cast<int64_t>(i) * d + j] -= s;
        }
    }
}

__global__ void chol_finish_kernel(int d, double *__restrict__ W)
{
    const int64_t n = static_cast<int64_t>(d) * d;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < n;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(idx / d), j = static_cast<int>(idx % d);
        if (j > i) W[idx] = 0.0;
    }
}

__global__ void scale_factor_kernel(int d, const double *L, const double *sigma, double c, double sdt,
                                    double r, double dt, int scheme, float *Lp, float *drift)
{
    const int64_t tot = static_cast<int64_t>(d) * (d + 1) / 2;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < tot;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        // packed lower triangle: row a at a(a+1)/2
        int a = static_cast<int>((sqrt(8.0 * static_cast<double>(idx) + 1.0) - 1.0) * 0.5);
        while (static_cast<int64_t>(a + 1) * (a + 2) / 2 <= idx) ++a;
        while (static_cast<int64_t>(a) * (a + 1) / 2 > idx) --a;
        const int k = static_cast<int>(idx - static_cast<int64_t>(a) * (a + 1) / 2);
        Lp[idx] = static_cast<float>(c * sdt * sigma[a] * L[static_cast<int64_t>(a) * d + k]);
    }
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < d; a += gridDim.x * blockDim.x)
        drift[a] = static_cast<float>(scheme == MC_LOG_EULER ? c * (r - 0.5 * sigma[a] * sigma[a]) * dt : r * dt);
}

}  // namespace

cudaError_t launch_cholesky(int d, const double *A, double *L, int *status, cudaStream_t s)
{
    if (d <= kCholSmallD) {
        cholesky_small_kernel<<<1, kCholSmallBlock, 0, s>>>(d, A, L, status);
        return cudaGetLastError();
    }
    const int64_t n = static_cast<int64_t>(d) * d;
    const int g = static_cast<int>(std::min<int64_t>((n + 255) / 256, 1024));
    chol_copy_kernel<<<g, 256, 0, s>>>(n, A, L, status);
    for (int k0 = 0; k0 < d; k0 += kCholNb) {
        const int nb = std::min(kCholNb, d - k0), rest = d - k0 - nb;
        chol_diag_kernel<<<1, 256, 0, s>>>(d, k0, nb, A, L, status);
        if (rest > 0) {
            chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(d, k0, nb, L);
            const int nbl = (rest + kCholNb - 1) / kCholNb;
            chol_update_kernel<<<nbl * (nbl + 1) / 2, 256, 0, s>>>(d, k0, nb, L);
        }
    }
    chol_finish_kernel<<<g, 256, 0, s>>>(d, L);
    return cudaGetLastError();
}

cudaError_t launch_scale_factor(int d, const double *L, const double *sigma, double c, double sdt,
                                double r, double dt, int scheme, float *Lpacked, float *drift,
                                cudaStream_t s)
{
    const int64_t tot = static_cast<int64_t>(d) * (d + 1) / 2;
    const int grid = static_cast<int>((tot + 255) / 256 > 1024 ? 1024 : (tot + 255) / 256);
    scale_factor_kernel<<<grid, 256, 0, s>>>(d, L, sigma, c, sdt, r, dt, scheme, Lpacked, drift);
    return cudaGetLastError();
}

}  // namespace gbmc
