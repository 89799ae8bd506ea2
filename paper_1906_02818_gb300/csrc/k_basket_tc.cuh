// Correlated-basket path kernel with the correlation contraction on the
// 5th-generation tensor cores (Sec. II.A.2: dW = sigma(X) Z for N stacked
// scenarios is a (paths x d) x (d x d) product; Sec. V.A: low-precision
// multiplies with FP32 accumulation).
//
// One CTA = 128 paths = 128 threads; thread t owns path row t of every tile
// and TMEM lane t.  Per step i:
//   1. each thread draws its row of Z_i (Philox4x32-10 + Box-Muller, fused in
//      registers), rounds it to BF16 / FP16 / E4M3 (E4M3 with a per-path,
//      per-step amax scale) and stores it in the 128B- (64B- for E4M3)
//      swizzled K-major shared-memory tile the MMA reads;
//   2. one thread issues tcgen05.mma: D[128 x 64] (TMEM, FP32) = Z_i Lq^T,
//      where Lq is the quantised Cholesky factor of the correlation (rows
//      scaled to the operand range), resident in shared memory;
//   3. every thread reads its row of D back (tcgen05.ld, 16 columns at a
//      time) and applies the FP32 step: y_n += drift_n + cs_n D_n (log-Euler on log2(S_n/S0_n)), or
//      S_n <- S_n (1 + r dt + cs_n D_n) (Euler), with cs_n folding
//      sqrt(dt) sigma_n and the operand scales.
// Z tiles are double-buffered so that drawing Z_{i+1} overlaps MMA_i.  All
// waits on the MMA's mbarrier are bounded; on expiry the CTA records an error
// word, stops simulating, frees its TMEM and still takes part in the
// reduction (the final block then reports NaN prices).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mc_kernels.cuh"
#include "tc_ptx.cuh"

namespace gbmc {

namespace tcb {

constexpr int kRows = 128;   // paths per tile = UMMA M
constexpr int kN = 64;       // assets (padded) = UMMA N = K
constexpr int kThreads = 128;

template <int PREC>
struct Layout {
    static constexpr int kElemBytes = PREC == MC_FP8E4M3 ? 1 : 2;
    static constexpr int kRowBytes = kN * kElemBytes;              // 128 or 64
    static constexpr int kTileBytes = kRows * kRowBytes;           // Z tile
    static constexpr int kBBytes = kN * kRowBytes;                 // factor tile
    static constexpr int kGroupBytes = 8 * kRowBytes;              // SBO
    static constexpr int kChunks = kRowBytes / 16;                 // 16-B chunks per row
    static constexpr int kPerChunk = 16 / kElemBytes;              // elements per chunk
    static constexpr int kKStep = PREC == MC_FP8E4M3 ? 32 : 16;    // UMMA K
    static constexpr int kMmas = kN / kKStep;
    static constexpr tc::Swizzle kSw = PREC == MC_FP8E4M3 ? tc::SW_64B : tc::SW_128B;
    // shared memory: [pad to 1024] Z0 | Z1 | B | mbarrier | tmem slot
    static constexpr int kSmem = 1024 + 2 * kTileBytes + kBBytes + 64;
    // byte offset of (row, chunk) inside a swizzled tile
    __device__ static __forceinline__ uint32_t chunk_off(int row, int chunk)
    {
        const int phys = PREC == MC_FP8E4M3 ? (chunk ^ ((row >> 1) & 3)) : (chunk ^ (row & 7));
        return static_cast<uint32_t>((row >> 3) * kGroupBytes + (row & 7) * kRowBytes + phys * 16);
    }
};

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if (PREC == MC_BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

__device__ __forceinline__ uint32_t pack4_e4m3(float a, float b, float c, float d)
{
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

struct Stats {
    float sum, umax, umin;
};

// Draws Z_i of path n (row `row`) into the tile at `tile`; returns the
// dequantisation factor of the row (1 unless E4M3).
template <int PREC, bool EXACT>
__device__ __forceinline__ float draw_row(uint32_t tile, int row, int i, int d, uint64_t n,
                                          const RoundKeys &rk, NormalReader &rd, bool valid)
{
    using Ly = Layout<PREC>;
    auto normal8 = [&](int c0, float (&z)[8]) {
        if (!valid) {
#pragma unroll
            for (int l = 0; l < 8; ++l) z[l] = 0.0f;
        } else if (EXACT) {
            const uint64_t q = static_cast<uint64_t>(i) * (kN / 4) + c0 / 4;
            const float4 a = normals4(q, n, rk), b = normals4(q + 1, n, rk);
            z[0] = a.x; z[1] = a.y; z[2] = a.z; z[3] = a.w; z[4] = b.x; z[5] = b.y; z[6] = b.z; z[7] = b.w;
        } else {
#pragma unroll
            for (int l = 0; l < 8; ++l)
                z[l] = (c0 + l < d) ? rd.get(static_cast<uint64_t>(i) * d + c0 + l) : 0.0f;
        }
    };
    if (PREC != MC_FP8E4M3) {
#pragma unroll
        for (int cb = 0; cb < Ly::kChunks; ++cb) {
            float z[8];
            normal8(cb * 8, z);
            st_shared_v4(tile + Ly::chunk_off(row, cb), pack2<PREC>(z[0], z[1]), pack2<PREC>(z[2], z[3]),
                         pack2<PREC>(z[4], z[5]), pack2<PREC>(z[6], z[7]));
        }
        return 1.0f;
    } else {
        float z[kN];
#pragma unroll
        for (int cb = 0; cb < kN / 8; ++cb) {
            float t[8];
            normal8(cb * 8, t);
#pragma unroll
            for (int l = 0; l < 8; ++l) z[cb * 8 + l] = t[l];
        }
        float amax = 0.0f;
#pragma unroll
        for (int j = 0; j < kN; ++j) amax = fmaxf(amax, fabsf(z[j]));
        const float s = amax > 0.0f ? 448.0f / amax : 1.0f;
#pragma unroll
        for (int cb = 0; cb < Ly::kChunks; ++cb) {
            const float *q = z + cb * 16;
            st_shared_v4(tile + Ly::chunk_off(row, cb), pack4_e4m3(q[0] * s, q[1] * s, q[2] * s, q[3] * s),
                         pack4_e4m3(q[4] * s, q[5] * s, q[6] * s, q[7] * s),
                         pack4_e4m3(q[8] * s, q[9] * s, q[10] * s, q[11] * s),
                         pack4_e4m3(q[12] * s, q[13] * s, q[14] * s, q[15] * s));
        }
        return amax > 0.0f ? amax / 448.0f : 1.0f;
    }
}

template <int PREC>
__device__ __forceinline__ void issue_mmas(uint32_t tmem_d, uint32_t ztile, uint32_t btile)
{
    using Ly = Layout<PREC>;
#pragma unroll
    for (int kk = 0; kk < Ly::kMmas; ++kk) {
        const uint64_t ad = tc::smem_desc(ztile + kk * 32, Ly::kGroupBytes, Ly::kSw);
        const uint64_t bd = tc::smem_desc(btile + kk * 32, Ly::kGroupBytes, Ly::kSw);
        if (PREC == MC_FP8E4M3) tc::mma_f8(tmem_d, ad, bd, tc::idesc_e4m3(kRows, kN), kk > 0 ? 1u : 0u);
        else tc::mma_f16(tmem_d, ad, bd, tc::idesc_f16(kRows, kN, PREC == MC_BF16), kk > 0 ? 1u : 0u);
    }
}

template <int PREC, int SCHEME, bool STATS, bool EXACT>
__global__ void __launch_bounds__(kThreads) basket_tc_kernel(const __grid_constant__ TcArgs a, const TcConst c)
{
    using Ly = Layout<PREC>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ AccSlot s_acc[(kThreads / 32) * MC_MAX_PAYOFFS * 2];
    __shared__ double s_red[32];

    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t zt[2] = {base, base + Ly::kTileBytes};
    const uint32_t bt = base + 2 * Ly::kTileBytes;
    const uint32_t mbar = bt + Ly::kBBytes;
    const uint32_t tslot = mbar + 16;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));

    for (int i = t; i < (kThreads / 32) * a.pay.n * 2; i += kThreads) s_acc[i] = 0.0f;
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_init(mbar + 8, 1);  // factor-tile load barrier
    }
    __syncthreads();
    // factor tile: one bulk (TMA) copy of the pre-swizzled image
    if (t == 0) {
        tc::mbar_arrive_expect_tx(mbar + 8, Ly::kBBytes);
        tc::bulk_g2s(bt, a.bimg, Ly::kBBytes, mbar + 8);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kN);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot_ptr;
    // CTA-uniform: every change goes through __syncthreads_or.
    // The factor tile's wait; a test request (a.stall = 1) redirects it to the
    // MMA barrier, to which no MMA has been committed yet, so it runs out.
    bool aborted = __syncthreads_or(tc::mbar_wait_bounded(mbar + 8 - 8 * a.stall, 0, a.wait_cap) ? 0 : 1) != 0;

    uint32_t phase = 0;
    const int M = a.run.steps, d = a.d;
    const float inv_m = 1.0f / static_cast<float>(M);
    const int64_t ntiles = (a.run.paths + kRows - 1) / kRows;
    const uint32_t row_taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t nl = tile * kRows + t;
        const bool valid = nl < a.run.paths;
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + (valid ? nl : 0));
        NormalReader rd;
        rd.init(n, a.run.rk);
        float x[kN];
#pragma unroll
        for (int j = 0; j < kN; ++j) x[j] = (SCHEME == MC_LOG_EULER) ? 0.0f : c.s0[j];
        Stats st{0.0f, -INFINITY, INFINITY};

        float deq_cur = 1.0f, deq_next = 1.0f;
        if (!aborted) {
            deq_cur = draw_row<PREC, EXACT>(zt[0], t, 0, d, n, a.run.rk, rd, valid);
            tc::fence_proxy_async();
        }
        __syncthreads();
        if (t == 0 && !aborted) {
            tc::fence_after_sync();
            issue_mmas<PREC>(tmem, zt[0], bt);
            tc::mma_commit(mbar);
        }
        for (int i = 0; i < M && !aborted; ++i) {
            if (i + 1 < M) {
                deq_next = draw_row<PREC, EXACT>(zt[(i + 1) & 1], t, i + 1, d, n, a.run.rk, rd, valid);
                tc::fence_proxy_async();
            }
            const bool ok = tc::mbar_wait_bounded(mbar, phase & 1u, a.wait_cap);
            ++phase;
            tc::fence_after_sync();
            // FP32 state update of step i, 16 accumulator columns at a time
            float u = 0.0f;
#pragma unroll
            for (int cc = 0; cc < kN / 16; ++cc) {
                float v[16];
                tc::tmem_ld16(row_taddr + cc * 16, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int l = 0; l < 16; ++l) {
                    const int j = cc * 16 + l;
                    const float dw = c.cs[j] * (v[l] * deq_cur);
                    if (SCHEME == MC_LOG_EULER) {
                        x[j] += c.drift[j] + dw;
                        if (STATS) u = fmaf(c.ws0[j], ex2_approx(x[j]), u);
                    } else {
                        x[j] = fmaf(x[j], c.drift[j] + dw, x[j]);
                        if (STATS) u = fmaf(c.w[j], x[j], u);
                    }
                }
            }
            tc::fence_before_sync();
            if (__syncthreads_or(ok ? 0 : 1)) aborted = true;
            if (t == 0 && i + 1 < M && !aborted) {
                tc::fence_after_sync();
                issue_mmas<PREC>(tmem, zt[(i + 1) & 1], bt);
                tc::mma_commit(mbar);
            }
            if (STATS) {
                st.sum += u;
                st.umax = fmaxf(st.umax, u);
                st.umin = fminf(st.umin, u);
            }
            deq_cur = deq_next;
        }
        float uT = 0.0f;
#pragma unroll
        for (int j = 0; j < kN; ++j) {
            if (SCHEME == MC_LOG_EULER) uT = fmaf(c.ws0[j], ex2_approx(x[j]), uT);
            else uT = fmaf(c.w[j], x[j], uT);
        }
        const float avg = st.sum * inv_m;
        const bool use = valid && !aborted;
        for (int p = 0; p < a.pay.n; ++p) {
            const float f = payoff_eval(a.pay.kind[p], a.pay.strike[p], a.pay.barrier[p], uT, avg, st.umax, st.umin);
            warp_accumulate(s_acc, a.pay.n, p, use ? f : 0.0f);
        }
        __syncthreads();
    }
    if (aborted && t == 0) {
        atomicExch(a.err, 1u);
        // drain before the shared memory and TMEM are released.  Without an
        // MMA (phase 0) the factor tile's copy may still be landing; after
        // one, that copy had landed, and the last committed MMA group may
        // still be running (every group is waited on once, `phase` counts
        // them, and only the last wait can have given up).  Bounded as ever.
        tc::mbar_wait_bounded(phase > 0 ? mbar : mbar + 8, phase > 0 ? (phase - 1) & 1u : 0u, a.wait_cap);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kN);
    }
    block_finish(s_acc, s_red, a.pay.n, a.red);
}

// Log-Euler with BF16 / FP16 operands: the running correlated increment
// D = sum_{steps <= i} Z Lq^T accumulates in TMEM across the steps (each
// step's MMA adds into it), so a thread keeps no per-asset state:
// log2(S_n(t_{i+1}) / S0_n) = (i + 1) drift_n + cs_n D_n is formed when a
// monitored statistic needs it and once at maturity.  One Z buffer; the
// small per-CTA footprint (64 TMEM columns, ~28 KB of shared memory, <= 64
// registers) lets 8 CTAs share an SM, which hides each CTA's MMA wait behind
// the others' normals.  Bounded waits as in basket_tc_kernel.
template <int PREC, bool STATS, bool EXACT>
__global__ void __launch_bounds__(kThreads, 8) basket_tc_acc_kernel(const __grid_constant__ TcArgs a, const TcConst c)
{
    using Ly = Layout<PREC>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ double s_red[32];
    // per-asset terms of the step s being observed, double-buffered by the
    // parity of s (written before the step's barrier, read after it):
    // BF16 w_n S0_n 2^{s drift_n}; FP16 s drift_n
    __shared__ __align__(16) float s_g[2][kN];

    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t zt = base, bt = base + Ly::kTileBytes;
    const uint32_t mbar = bt + Ly::kBBytes, tslot = mbar + 16;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));
    // per-warp payoff slots after the barriers, sized by the payoff count at
    // launch (a static array for 32 payoffs would cost an SM its eighth CTA)
    AccSlot *s_acc = reinterpret_cast<AccSlot *>(smem_raw + (mbar + 32 - raw));

    for (int i = t; i < (kThreads / 32) * a.pay.n * 2; i += kThreads) s_acc[i] = 0.0f;
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_init(mbar + 8, 1);
    }
    __syncthreads();
    if (t == 0) {
        tc::mbar_arrive_expect_tx(mbar + 8, Ly::kBBytes);
        tc::bulk_g2s(bt, a.bimg, Ly::kBBytes, mbar + 8);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kN);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot_ptr;
    // The factor tile's wait; a test request (a.stall = 1) redirects it to the
    // MMA barrier, to which no MMA has been committed yet, so it runs out.
    bool aborted = __syncthreads_or(tc::mbar_wait_bounded(mbar + 8 - 8 * a.stall, 0, a.wait_cap) ? 0 : 1) != 0;

    uint32_t phase = 0;
    const int M = a.run.steps, d = a.d;
    const float inv_m = 1.0f / static_cast<float>(M);
    const int64_t ntiles = (a.run.paths + kRows - 1) / kRows;
    const uint32_t row_taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    // basket value of this thread's path after s steps, from its accumulator
    // row: sum_n w_n S0_n 2^{s drift_n + cs_n D_n}; BF16 (cs_n = 1, folded into
    // the operand) as sum_n g_n 2^{D_n} with g_n = w_n S0_n 2^{s drift_n} from
    // s_g[s & 1]; FP16 with s drift_n from s_g[s & 1]
    constexpr bool kFold = PREC == MC_BF16;
    auto basket = [&](int buf) {
        float u = 0.0f;
        const float4 *g4 = reinterpret_cast<const float4 *>(s_g[buf]);
#pragma unroll
        for (int cc = 0; cc < kN / 16; ++cc) {
            float v[16];
            tc::tmem_ld16(row_taddr + cc * 16, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 g = g4[cc * 4 + q];
                const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                for (int l4 = 0; l4 < 4; ++l4) {
                    const int l = 4 * q + l4, j = cc * 16 + l;
                    u = kFold ? fmaf(gv[l4], ex2_approx(v[l]), u)
                              : fmaf(c.ws0[j], ex2_approx(fmaf(c.cs[j], v[l], gv[l4])), u);
                }
            }
        }
        return u;
    };
    auto set_g = [&](int steps) {
        if (t < kN)
            s_g[steps & 1][t] = kFold ? c.ws0[t] * ex2_approx(static_cast<float>(steps) * c.drift[t])
                                      : static_cast<float>(steps) * c.drift[t];
    };

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t nl = tile * kRows + t;
        const bool valid = nl < a.run.paths;
        const uint64_t n = static_cast<uint64_t>(a.run.path_offset + (valid ? nl : 0));
        NormalReader rd;
        rd.init(n, a.run.rk);
        Stats st{0.0f, -INFINITY, INFINITY};
        bool ok = true;
        for (int i = 0; i < M; ++i) {
            // s_g[(i + 1) & 1] was last read before the previous step's barrier
            if (STATS || i + 1 == M) set_g(i + 1);
            if (!aborted) draw_row<PREC, EXACT>(zt, t, i, d, n, a.run.rk, rd, valid);
            tc::fence_proxy_async();
            tc::fence_before_sync();  // this thread's accumulator reads precede the next MMA
            if (__syncthreads_or(ok ? 0 : 1)) aborted = true;
            if (aborted) break;
            if (t == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int kk = 0; kk < Ly::kMmas; ++kk) {
                    const uint64_t ad = tc::smem_desc(zt + kk * 32, Ly::kGroupBytes, Ly::kSw);
                    const uint64_t bd = tc::smem_desc(bt + kk * 32, Ly::kGroupBytes, Ly::kSw);
                    tc::mma_f16(tmem, ad, bd, tc::idesc_f16(kRows, kN, PREC == MC_BF16), (i > 0 || kk > 0) ? 1u : 0u);
                }
                tc::mma_commit(mbar);
            }
            ok = tc::mbar_wait_bounded(mbar, phase & 1u, a.wait_cap);
            ++phase;
            tc::fence_after_sync();
            // the Z buffer is free again (the MMA completed); the accumulator holds steps 0..i
            if (STATS && __all_sync(0xffffffffu, ok)) {
                const float u = basket((i + 1) & 1);
                st.sum += u;
                st.umax = fmaxf(st.umax, u);
                st.umin = fminf(st.umin, u);
            }
        }
        if (__syncthreads_or(ok ? 0 : 1)) aborted = true;
        const float uT = aborted ? 0.0f : basket(M & 1);
        const float avg = st.sum * inv_m;
        const bool use = valid && !aborted;
        for (int p = 0; p < a.pay.n; ++p) {
            const float f = payoff_eval(a.pay.kind[p], a.pay.strike[p], a.pay.barrier[p], uT, avg, st.umax, st.umin);
            warp_accumulate(s_acc, a.pay.n, p, use ? f : 0.0f);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (aborted && t == 0) {
        atomicExch(a.err, 1u);
        // drain before the shared memory and TMEM are released.  Without an
        // MMA (phase 0) the factor tile's copy may still be landing; after
        // one, that copy had landed, and the last committed MMA group may
        // still be running (every group is waited on once, `phase` counts
        // them, and only the last wait can have given up).  Bounded as ever.
        tc::mbar_wait_bounded(phase > 0 ? mbar : mbar + 8, phase > 0 ? (phase - 1) & 1u : 0u, a.wait_cap);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kN);
    }
    block_finish(s_acc, s_red, a.pay.n, a.red);
}

// Factor tile for the MMA's B operand: row n = Lrho[n][0..63] (zero above
// the diagonal and beyond d), scaled by s_n (E4M3: 448 / max_k |Lrho[n][k]|;
// BF16: c sqrt(dt) sigma_n; FP16: 1), rounded to the operand type, at its
// swizzled position.  Also the FP32 per-column scale
// cs_n = c sqrt(dt) sigma_n / s_n and the drift.
template <int PREC>
__global__ void tc_prep_kernel(int d, const double *L, const double *sigma, double cfac, double sdt, double r,
                               double dt, int scheme, uint8_t *bimg, float *cs, float *drift)
{
    using Ly = Layout<PREC>;
    const int nrow = threadIdx.x;
    if (nrow >= kN) return;
    double amax = 0.0;
    for (int k = 0; k < kN; ++k) {
        const double v = (nrow < d && k <= nrow) ? L[static_cast<int64_t>(nrow) * d + k] : 0.0;
        amax = fmax(amax, fabs(v));
    }
    // BF16: the row carries its column scale c sqrt(dt) sigma_n (bf16 keeps
    // the full FP32 exponent range), so the accumulator holds log2-price
    // increments and cs_n = 1.
    // (sigma_n = 0: a zero row)
    const double colscale = nrow < d ? cfac * sdt * sigma[nrow] : 0.0;
    const double s = (PREC == MC_FP8E4M3 && amax > 0.0) ? 448.0 / amax : (PREC == MC_BF16 ? colscale : 1.0);
    for (int k = 0; k < kN; ++k) {
        const double v = (nrow < d && k <= nrow) ? L[static_cast<int64_t>(nrow) * d + k] * s : 0.0;
        const uint32_t off = Ly::chunk_off(nrow, k / Ly::kPerChunk) + (k % Ly::kPerChunk) * Ly::kElemBytes;
        // rounded through binary32, like the normals (one rule for both operands)
        const float fv = static_cast<float>(v);
        if (PREC == MC_BF16) {
            *reinterpret_cast<__nv_bfloat16 *>(bimg + off) = __float2bfloat16_rn(fv);
        } else if (PREC == MC_FP16) {
            *reinterpret_cast<__half *>(bimg + off) = __float2half_rn(fv);
        } else {
            uint16_t pr;
            asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(pr) : "f"(0.0f), "f"(fv));
            bimg[off] = static_cast<uint8_t>(pr & 0xFFu);
        }
    }
    if (nrow < d) {
        cs[nrow] = PREC == MC_BF16 ? 1.0f : static_cast<float>(cfac * sdt * sigma[nrow] / s);
        drift[nrow] = static_cast<float>(scheme == MC_LOG_EULER ? cfac * (r - 0.5 * sigma[nrow] * sigma[nrow]) * dt
                                                                : r * dt);
    } else {
        cs[nrow] = 0.0f;
        drift[nrow] = 0.0f;
    }
}

}  // namespace tcb

template <int PREC, int SCHEME>
const void *basket_tc_select(const TcArgs &a, int *smem)
{
    const bool stats = a.pay.need_avg || a.pay.need_max || a.pay.need_min;
    const bool exact = a.d == tcb::kN;
    if constexpr (PREC != MC_FP8E4M3 && SCHEME == MC_LOG_EULER) {
        // TMEM running sum: Z tile + factor tile + barriers + payoff slots
        // (~27 KB with the static arrays and the per-block reservation: at
        // most 8 CTAs, 8 x 64 TMEM columns, share an SM)
        *smem = 1024 + tcb::Layout<PREC>::kTileBytes + tcb::Layout<PREC>::kBBytes + 32 +
                (tcb::kThreads / 32) * a.pay.n * 2 * static_cast<int>(sizeof(AccSlot));
        if (stats)
            return exact ? reinterpret_cast<const void *>(&tcb::basket_tc_acc_kernel<PREC, true, true>)
                         : reinterpret_cast<const void *>(&tcb::basket_tc_acc_kernel<PREC, true, false>);
        return exact ? reinterpret_cast<const void *>(&tcb::basket_tc_acc_kernel<PREC, false, true>)
                     : reinterpret_cast<const void *>(&tcb::basket_tc_acc_kernel<PREC, false, false>);
    }
    *smem = tcb::Layout<PREC>::kSmem;
    if (stats)
        return exact ? reinterpret_cast<const void *>(&tcb::basket_tc_kernel<PREC, SCHEME, true, true>)
                     : reinterpret_cast<const void *>(&tcb::basket_tc_kernel<PREC, SCHEME, true, false>);
    return exact ? reinterpret_cast<const void *>(&tcb::basket_tc_kernel<PREC, SCHEME, false, true>)
                 : reinterpret_cast<const void *>(&tcb::basket_tc_kernel<PREC, SCHEME, false, false>);
}

template <int PREC>
cudaError_t tc_prep(int d, const double *L, const double *sigma, double cfac, double sdt, double r, double dt,
                    int scheme, uint8_t *bimg, float *cs, float *drift, cudaStream_t s)
{
    tcb::tc_prep_kernel<PREC><<<1, tcb::kN, 0, s>>>(d, L, sigma, cfac, sdt, r, dt, scheme, bimg, cs, drift);
    return cudaGetLastError();
}

#define GBMC_INSTANTIATE_TC(PREC)                                                                         \
    template const void *basket_tc_select<PREC, MC_LOG_EULER>(const TcArgs &a, int *smem);               \
    template const void *basket_tc_select<PREC, MC_EULER>(const TcArgs &a, int *smem);                   \
    template cudaError_t tc_prep<PREC>(int, const double *, const double *, double, double, double, double, \
                                       int, uint8_t *, float *, float *, cudaStream_t);

}  // namespace gbmc
