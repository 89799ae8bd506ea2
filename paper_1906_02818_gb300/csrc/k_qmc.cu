// Randomised quasi-Monte Carlo (Sec. IV, the QRNG / Sobol discussion, and
// the Sobol basket experiment of Sec. VI.D): correlated GBM baskets driven by
// a Sobol sequence instead of Philox normals.
//   * Sobol construction (host, below): dimension 1 is van der Corput;
//     dimension j >= 2 takes the (j-1)-th primitive polynomial over GF(2)
//     (by degree, then by value), initial direction integers m_1..m_s = 1 and
//     the Bratley-Fox recurrence; V_k = m_k 2^(32-k).
//   * Point n (natural order) of dimension j: XOR of V_j[k] over the set bits
//     k of n.  Replication r XORs every point of dimension j with word j of
//     Philox stream 6 * 2^56 + r (a random digital shift), so each
//     replication is an unbiased estimate and their spread gives the error.
//   * Normal a of step i is the cosine branch of Box-Muller on dimensions
//     2 (i d + a) and 2 (i d + a) + 1 (the paper's 32 dimensions for 16
//     assets); 2 d M <= 64.
//   * The step, statistics and payoffs are those of the FP32 basket path:
//     log-Euler on log2(S/S0) (or Euler on S) with Lhat = c sqrt(dt)
//     diag(sigma) Lrho.
// One thread per point; per replication (grid.y) the block sums its payoffs
// and adds them to an FP64 total.
#include "mc_kernels.cuh"

namespace gbmc {

namespace {

constexpr int kBlock = 256;
constexpr int kDmax = kQmcMaxAssets;

template <int SCHEME, bool STATS>
__global__ void __launch_bounds__(kBlock) qmc_kernel(const __grid_constant__ QmcArgs a, const QmcConst c)
{
    __shared__ uint32_t s_v[kQmcMaxDims][32];
    __shared__ uint32_t s_shift[kQmcMaxDims];
    __shared__ AccSlot s_acc[(kBlock / 32) * MC_MAX_PAYOFFS * 2];
    const int t = threadIdx.x, nd = a.ndim, np = a.pay.n;
    const int64_t rep = blockIdx.y;
    for (int i = t; i < nd * 32; i += kBlock) s_v[i / 32][i % 32] = c.V[i / 32][i % 32];
    if (t * 4 < nd) {  // digital shift of this replication: Philox words of stream 6 * 2^56 + r
        const uint64_t stream = (uint64_t(6) << 56) | static_cast<uint64_t>(rep);
        const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(t), 0u, static_cast<uint32_t>(stream),
                                                 static_cast<uint32_t>(stream >> 32)),
                                      a.rk);
        const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
        for (int l = 0; l < 4 && 4 * t + l < nd; ++l) s_shift[4 * t + l] = w4[l];
    }
    for (int i = t; i < (kBlock / 32) * np * 2; i += kBlock) s_acc[i] = 0.0f;
    __syncthreads();

    const int d = a.d, M = a.steps;
    const float inv_m = 1.0f / static_cast<float>(M);
    // block-uniform trip count: every lane takes part in the warp reductions
    for (int64_t base = blockIdx.x * static_cast<int64_t>(kBlock); base < a.npts;
         base += static_cast<int64_t>(gridDim.x) * kBlock) {
        const int64_t pt = base + t;
        const bool valid = pt < a.npts;
        const uint64_t n = static_cast<uint64_t>(a.n0 + (valid ? pt : 0));
        float x[kDmax];
#pragma unroll
        for (int j = 0; j < kDmax; ++j) x[j] = (SCHEME == MC_LOG_EULER) ? 0.0f : c.s0[j];
        float sum = 0.0f, umax = -INFINITY, umin = INFINITY, u = 0.0f;
        for (int i = 0; i < M; ++i) {
            float z[kDmax];
#pragma unroll
            for (int k = 0; k < kDmax; ++k) {
                z[k] = 0.0f;
                if (k < d) {
                    const int j = 2 * (i * d + k);
                    uint32_t w1 = s_shift[j], w2 = s_shift[j + 1];
                    for (uint64_t m = n; m; m &= m - 1) {
                        const int b = __ffsll(static_cast<long long>(m)) - 1;
                        w1 ^= s_v[j][b];
                        w2 ^= s_v[j + 1][b];
                    }
                    float z1;
                    box_muller(w1, w2, z[k], z1);
                }
            }
#pragma unroll
            for (int q = 0; q < kDmax; ++q) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k <= q; ++k) acc = fmaf(c.L[q * (q + 1) / 2 + k], z[k], acc);
                if (SCHEME == MC_LOG_EULER) x[q] += c.drift[q] + acc;
                else x[q] = fmaf(x[q], c.drift[q] + acc, x[q]);
            }
            if (STATS || i == M - 1) {
                u = 0.0f;
#pragma unroll
                for (int q = 0; q < kDmax; ++q)
                    u = (SCHEME == MC_LOG_EULER) ? fmaf(c.ws0[q], ex2_approx(x[q]), u) : fmaf(c.w[q], x[q], u);
                sum += u;
                umax = fmaxf(umax, u);
                umin = fminf(umin, u);
            }
        }
        for (int p = 0; p < np; ++p) {
            const float f = payoff_eval(a.pay.kind[p], a.pay.strike[p], a.pay.barrier[p], u, sum * inv_m, umax, umin);
            warp_accumulate(s_acc, np, p, valid ? f : 0.0f);
        }
    }
    __syncthreads();
    for (int p = t; p < np; p += kBlock) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += s_acc[(w * np + p) * 2];
        atomicAdd(a.sums + rep * np + p, s);
    }
}

template <int SCHEME, bool STATS>
const void *fn() { return reinterpret_cast<const void *>(&qmc_kernel<SCHEME, STATS>); }

const void *select(const QmcArgs &a)
{
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    if (a.scheme == MC_LOG_EULER) return stats ? fn<MC_LOG_EULER, true>() : fn<MC_LOG_EULER, false>();
    return stats ? fn<MC_EULER, true>() : fn<MC_EULER, false>();
}

// Degree of a GF(2) polynomial given as its coefficient bits.
int degree(uint32_t p)
{
    int s = -1;
    for (; p; p >>= 1) ++s;
    return s;
}

// The multiplicative order of x modulo p (degree s >= 1, p(0) = 1): the
// smallest e >= 1 with x^e = 1, found by stepping through the powers of x.
uint32_t order_of_x(uint32_t p, int s)
{
    const uint32_t top = 1u << s, mask = top - 1u;
    uint32_t r = 1u;
    for (uint32_t e = 1; e <= mask + 1u; ++e) {
        r <<= 1;  // times x
        if (r & top) r = (r ^ p) & mask;
        if (r == 1u) return e;
    }
    return 0;
}

}  // namespace

// Direction words of dimensions 0 .. ndim - 1, by the recurrence on the words
// themselves: V_k = V_{k-s} ^ (V_{k-s} >> s) ^ sum_i a_i V_{k-i} (k > s),
// V_k = 2^(32-k) for k <= s (m_k = 1), a_i the coefficient of x^(s-i).
void qmc_directions(int ndim, uint32_t (*V)[32])
{
    for (int k = 1; k <= 32; ++k) V[0][k - 1] = 0x80000000u >> (k - 1);
    uint32_t poly = 2;
    for (int j = 1; j < ndim; ++j) {
        int s;
        do {  // next primitive polynomial: odd, x of order 2^s - 1
            ++poly;
            s = degree(poly);
        } while (!(poly & 1u) || order_of_x(poly, s) != (1u << s) - 1u);
        uint32_t *v = V[j];
        for (int k = 1; k <= 32; ++k) {
            if (k <= s) {
                v[k - 1] = 0x80000000u >> (k - 1);
                continue;
            }
            uint32_t w = v[k - s - 1] ^ (v[k - s - 1] >> s);
            for (int i = 1; i < s; ++i) w ^= ((poly >> (s - i)) & 1u) ? v[k - i - 1] : 0u;
            v[k - 1] = w;
        }
    }
}

cudaError_t launch_qmc(const QmcArgs &a, const QmcConst &c, int grid, cudaStream_t s)
{
    void *args[] = {const_cast<QmcArgs *>(&a), const_cast<QmcConst *>(&c)};
    return cudaLaunchKernel(select(a), dim3(grid, a.reps), dim3(kBlock), args, 0, s);
}

int qmc_occupancy(const QmcArgs &a)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select(a), kBlock, 0) != cudaSuccess) return 0;
    return nb;
}

int qmc_block() { return kBlock; }

}  // namespace gbmc
