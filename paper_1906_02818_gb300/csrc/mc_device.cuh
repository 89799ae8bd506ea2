// Device building blocks shared by the path kernels: the keyed counter-based
// generator (Sec. IV.A), the Box-Muller transform (Sec. VI.D), payoffs on the
// monitored underlying (Sec. I.A.2) and the warp / block / cross-block
// reduction that ends in the FP64 estimator of Eq. 3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mc.h"

namespace gbmc {

constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with the round multipliers, xor of the high halves with the other counter
// words and the round key, and a Weyl bump of the key between rounds.  The
// ten round keys are formed once per launch on the host and read from the
// kernel's parameter block (constant bank), so no round spends an
// instruction or a register on the key schedule.
// ---------------------------------------------------------------------------
struct RoundKeys {
    uint32_t k[20];  // round r: (k[2r], k[2r + 1]) = (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85)
};

__host__ __device__ inline RoundKeys round_keys(uint32_t k0, uint32_t k1)
{
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        rk.k[2 * r + 1] = k1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c = make_uint4(hi1 ^ c.y ^ rk.k[2 * round], lo1, hi0 ^ c.w ^ rk.k[2 * round + 1], lo0);
    }
    return c;
}

// u = (floor(x / 2^9) + 1/2) 2^-23 in [2^-24, 1 - 2^-24], exact in binary32:
// the bits of 1 + floor(x/2^9) 2^-23 minus (1 - 2^-24) (Sterbenz: exact).
__device__ __forceinline__ float u01(uint32_t x)
{
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.99999994039535522f;
}

// Box-Muller on one pair of words: z0 = r cos(2 pi u_b), z1 = r sin(2 pi u_b),
// r = sqrt(-2 ln u_a), evaluated with the SFU's approximate instructions
// (lg2, sqrt, sin, cos: one issue slot each).  The angle is taken as
// theta = 2 pi (u_b - 1/2) in (-pi, pi), the range where sin/cos.approx are
// most accurate, and the sign flip (cos(theta) = -cos(2 pi u_b), likewise
// sin) is folded into r.  theta comes from one FMA on f = 1 + floor(b/2^9)
// 2^-23 (the bits of u01 before its subtraction): f fl(2 pi) - fl(3 pi),
// within 3.5e-7 of 2 pi (u_b - 1/2) over all 2^23 values of f (two roundings
// of the constants, one of the FMA) and inside (-pi, pi).  -2 ln u_a is
// clamped at 0: lg2.approx has an absolute error near 2^-22 close to u = 1.
// The per-normal absolute error is a few 1e-6, except for u_a within ~1e-6
// of 1, where r < ~1.5e-3 is off by at most sqrt(1.39 * 2^-22) ~ 6e-4.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1)
{
    const float ua = u01(a);
    // -2 ln u = -2 ln(2) log2(u)
    const float r2 = fmaxf(-1.3862943611198906f * lg2_approx(ua), 0.0f);
    const float nrad = -sqrt_approx(r2);
    const float theta = fmaf(__uint_as_float(0x3F800000u | (b >> 9)), 6.2831854820251465f, -9.42477798461914f);
    z0 = nrad * cos_approx(theta);
    z1 = nrad * sin_approx(theta);
}

// Packed FP32 pairs (fma.rn.f32x2 and friends: each lane an ordinary FP32
// operation; low half = the even element).
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 fadd2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float lo_of(f32x2 v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float hi_of(f32x2 v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }
// The four normals of block q of stream (path) n.
__device__ __forceinline__ float4 normals4(uint64_t q, uint64_t n, const RoundKeys &rk)
{
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                             static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32)),
                                  rk);
    float4 z;
    box_muller(x.x, x.y, z.x, z.y);
    box_muller(x.z, x.w, z.z, z.w);
    return z;
}

// Sequential reader of normal j of one stream, regenerating a block only when
// j leaves the cached one (warp-uniform when all lanes are at the same j).
struct NormalReader {
    uint64_t n;
    const RoundKeys *rk;
    uint64_t q;
    float4 z;
    __device__ __forceinline__ void init(uint64_t stream, const RoundKeys &keys)
    {
        n = stream; rk = &keys; q = ~0ull;
    }
    __device__ __forceinline__ float get(uint64_t j)
    {
        const uint64_t qj = j >> 2;
        if (qj != q) { q = qj; z = normals4(qj, n, *rk); }
        const uint32_t l = static_cast<uint32_t>(j) & 3u;
        return l == 0 ? z.x : (l == 1 ? z.y : (l == 2 ? z.z : z.w));
    }
};

// ---------------------------------------------------------------------------
// Payoffs (undiscounted) on the monitored statistics of U.
// ---------------------------------------------------------------------------
struct PayoffSet {
    int n;
    int need_avg;   // some payoff uses the arithmetic average
    int need_max;   // some payoff uses the running maximum
    int need_min;   // some payoff uses the running minimum
    int kind[MC_MAX_PAYOFFS];
    float strike[MC_MAX_PAYOFFS];
    float barrier[MC_MAX_PAYOFFS];
};

__device__ __forceinline__ float payoff_eval(int kind, float K, float H, float uT, float avg,
                                             float umax, float umin)
{
    const float call = fmaxf(uT - K, 0.0f), put = fmaxf(K - uT, 0.0f);
    const bool up = umax >= H, down = umin <= H;
    switch (kind) {
    case MC_CALL: return call;
    case MC_PUT: return put;
    case MC_ASIAN_CALL: return fmaxf(avg - K, 0.0f);
    case MC_ASIAN_PUT: return fmaxf(K - avg, 0.0f);
    case MC_UO_CALL: return up ? 0.0f : call;
    case MC_UI_CALL: return up ? call : 0.0f;
    case MC_UO_PUT: return up ? 0.0f : put;
    case MC_UI_PUT: return up ? put : 0.0f;
    case MC_DO_CALL: return down ? 0.0f : call;
    case MC_DI_CALL: return down ? call : 0.0f;
    case MC_DO_PUT: return down ? 0.0f : put;
    case MC_DI_PUT: return down ? put : 0.0f;
    default: return 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Reduction.  Each warp owns a slot per payoff in shared memory; after every
// grid-stride iteration the warp's 32 payoffs (and squares) are summed in
// FP32 with shuffles and lane 0 adds them to its FP64 slot (fixed order:
// deterministic; FP64 so that a slot's error does not grow with the paths
// per thread).  At block end the warp slots are summed into one (sum f,
// sum f^2) pair per payoff, written to the block's partials in FP32.  The
// last block to finish (atomic ticket, no spin-wait) adds all block partials
// with compensated (Kahan) FP64 sums, forms mean and standard error,
// discounts and writes the results, then resets the ticket for the next
// launch.
// ---------------------------------------------------------------------------
using AccSlot = double;  // per-warp payoff slot in shared memory

// Compensated summation (Kahan): s + c carries the sum to about one FP64
// rounding whatever the number of terms.
struct KahanSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        const double y = x - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
struct ReduceArgs {
    float *partials;        // [gridDim.x][n_payoff][2]
    unsigned int *ticket;   // zero on entry to the launch, reset by the last block
    mc_result *out;         // [n_payoff]
    int64_t paths;
    double disc;
    const unsigned int *err;  // optional: non-zero means a CTA gave up; results become NaN
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds this warp's 32 payoff values to s_acc[warp][p][*].
__device__ __forceinline__ void warp_accumulate(AccSlot *s_acc, int np, int p, float f)
{
    const float a = warp_sum(f), b = warp_sum(f * f);
    if ((threadIdx.x & 31) == 0) {
        AccSlot *slot = s_acc + ((threadIdx.x >> 5) * np + p) * 2;
        slot[0] += static_cast<double>(a);
        slot[1] += static_cast<double>(b);
    }
}

// Called by every thread of the block after its last path.  s_acc holds
// nwarps*np*2 slots; s_red is scratch for 32 doubles.
__device__ inline void block_finish(AccSlot *s_acc, double *s_red, int np, const ReduceArgs &ra)
{
    const int nwarps = blockDim.x >> 5;
    __syncthreads();
    for (int i = threadIdx.x; i < np * 2; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += s_acc[w * np * 2 + i];
        ra.partials[static_cast<size_t>(blockIdx.x) * np * 2 + i] = static_cast<float>(s);
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int s_last;
    if (threadIdx.x == 0) s_last = (atomicAdd(ra.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Sums of all blocks' partials in FP64, in a fixed order (deterministic):
    // few payoffs: one warp per payoff, its lanes striding over the blocks;
    // many payoffs: one thread per payoff, over the blocks in order (each
    // block's row of partials is then read coalesced across the threads).
    const int nb = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    (void)s_red;
    const bool wide = np >= 32;
    const int first = wide ? static_cast<int>(threadIdx.x) : warp;
    const int stride = wide ? static_cast<int>(blockDim.x) : nwarps;
    for (int p = first; p < np; p += stride) {
        KahanSum k0, k1;
        double t0, t1;
        if (wide) {
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                const float2 q = *reinterpret_cast<const float2 *>(ra.partials + static_cast<size_t>(b) * np * 2 + p * 2);
                k0.add(static_cast<double>(q.x));
                k1.add(static_cast<double>(q.y));
            }
            t0 = k0.s;
            t1 = k1.s;
        } else {
            for (int b = lane; b < nb; b += 32) {
                const float *q = ra.partials + static_cast<size_t>(b) * np * 2 + p * 2;
                k0.add(static_cast<double>(q[0]));
                k1.add(static_cast<double>(q[1]));
            }
            // the 32 lanes' compensated sums, then a pairwise (shuffle tree) sum
            t0 = warp_sum_d(k0.s - k0.c);
            t1 = warp_sum_d(k1.s - k1.c);
        }
        if (wide || lane == 0) {
            const bool bad = ra.err && *reinterpret_cast<const volatile unsigned int *>(ra.err) != 0u;
            const double N = static_cast<double>(ra.paths);
            const double mean = t0 / N, m2 = t1 / N;
            const double var = fmax(m2 - mean * mean, 0.0);
            mc_result res;
            res.price = bad ? __longlong_as_double(0x7ff8000000000000ll) : ra.disc * mean;
            res.se = bad ? res.price : (ra.paths > 1 ? ra.disc * sqrt(var / (N - 1.0)) : 0.0);
            ra.out[p] = res;
        }
    }
    if (threadIdx.x == 0) *ra.ticket = 0u;
}

}  // namespace gbmc
