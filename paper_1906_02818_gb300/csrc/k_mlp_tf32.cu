// Training GEMMs of the pricing surrogate on the 5th-generation tensor cores
// (back-propagation through the network, Sec. I.A.3, on the DNN-layer
// analogue of Sec. III.C): C[M x N] = A[M x K] B[N x K]^T with both operands
// K-major FP32 in global memory, FP32 accumulation in tensor memory.
//
// Three-pass TF32 ("3xTF32"): each operand is split into hi = x with its low
// 13 mantissa bits cleared (exact in TF32) and lo = x - hi (exact in FP32,
// read by the tensor core to TF32), and the product is accumulated as
// hi*hi + hi*lo + lo*hi; the dropped lo*lo term and the TF32 reading of lo
// leave a relative error near 2^-21 per product, FP32-like.
//
// One CTA computes a 128 x 64 tile.  Eight loader warps load their share of
// each 32-wide K chunk two chunks ahead into registers and stage it (A: 128
// rows, B: 64 rows, 128-byte rows, 128-byte swizzle) as hi and lo planes in
// one of two stages, then arrive on the stage's `full` mbarrier; one lane of
// a ninth warp waits on it, issues the chunk's 12 MMAs (4 K-steps of 8, 3
// passes) and commits them to the stage's `empty` mbarrier, on which the
// loaders wait before refilling the stage.  The epilogue (loader warps)
// reads the accumulator (TMEM lane = row), writes the transposed output from
// registers, stages the tile in shared memory for coalesced row-major
// stores, and applies one of:
//   FWD: v = acc + b; Z = v; H = silu(v); Ht = H^T        (forward layer)
//   BWD: dZ = acc * silu'(Zin); dZt = dZ^T                (dH = dZ_next W)
//   PART: P[slice] = acc                                   (split-K, dW^T)
// Every mbarrier wait is bounded; on expiry the CTA sets *err and skips the
// remaining work (its outputs are then undefined and the call fails).
#include "mc_kernels.cuh"
#include "mlp.cuh"
#include "tc_ptx.cuh"

namespace gbmc {
namespace mtf {

constexpr int kBM = 128, kBN = 64, kBK = 32, kThreads = 256;
constexpr int kATile = kBM * kBK * 4;                  // 16 KB per plane
constexpr int kBTile = kBN * kBK * 4;                  // 8 KB per plane
constexpr int kStage = 2 * kATile + 2 * kBTile;        // hi + lo of A and B
constexpr int kSmem = 1024 + 2 * kStage + 64;          // align pad, 2 stages, barriers + TMEM slot

// Byte offset of 16-byte chunk `ch` (0..7) of row `row` in a 128-byte-row,
// 128-byte-swizzled K-major tile (8-row groups of 1024 bytes).
__device__ __forceinline__ uint32_t sw128(int row, int ch)
{
    return static_cast<uint32_t>((row >> 3) * 1024 + (row & 7) * 128 + ((ch ^ (row & 7)) << 4));
}

// Instruction descriptor of kind::tf32: F32 accumulate, A and B TF32, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void split(float x, float &hi, float &lo)
{
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

__device__ __forceinline__ void st4(uint32_t addr, float a, float b, float c, float d)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

constexpr int kALoads = kBM * 8 / kThreads;  // float4 of A per thread and chunk
constexpr int kBLoads = kBN * 8 / kThreads;  // float4 of B per thread and chunk
constexpr int kCStride = kBN + 4;            // row stride of the staged output tile (floats)

// One K chunk's share of this thread: A rows (idx >> 3), 16-byte column
// chunk (idx & 7), idx = threadIdx.x + i kThreads.
struct Frag {
    float4 a[kALoads];
    float4 b[kBLoads];
};

// K columns kk .. kk + 3 of row gr (zero past nrows or K).
__device__ __forceinline__ float4 ld_chunk(const float *__restrict__ X, int64_t ld, int64_t nrows, int K, int64_t gr,
                                           int kk)
{
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr < nrows && kk + 3 < K) {
        v = __ldg(reinterpret_cast<const float4 *>(X + gr * ld + kk));
    } else if (gr < nrows && kk < K) {  // ragged end of K: element loads
        const float *q = X + gr * ld + kk;
        v.x = q[0];
        if (kk + 1 < K) v.y = q[1];
        if (kk + 2 < K) v.z = q[2];
    }
    return v;
}

__device__ __forceinline__ void load_frag(Frag &f, const TfGemmArgs &a, int64_t m0, int n0, int ke, int k0)
{
#pragma unroll
    for (int i = 0; i < kALoads; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        f.a[i] = ld_chunk(a.A, a.lda, a.M, ke, m0 + (idx >> 3), k0 + 4 * (idx & 7));
    }
#pragma unroll
    for (int i = 0; i < kBLoads; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        f.b[i] = ld_chunk(a.B, a.ldb, a.N, ke, n0 + (idx >> 3), k0 + 4 * (idx & 7));
    }
}

__device__ __forceinline__ void store4(const float4 v, uint32_t hi_base, uint32_t lo_base, int idx)
{
    float h0, h1, h2, h3, l0, l1, l2, l3;
    split(v.x, h0, l0);
    split(v.y, h1, l1);
    split(v.z, h2, l2);
    split(v.w, h3, l3);
    const uint32_t off = sw128(idx >> 3, idx & 7);
    st4(hi_base + off, h0, h1, h2, h3);
    st4(lo_base + off, l0, l1, l2, l3);
}

__device__ __forceinline__ void store_frag(const Frag &f, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo)
{
#pragma unroll
    for (int i = 0; i < kALoads; ++i) store4(f.a[i], a_hi, a_lo, threadIdx.x + i * kThreads);
#pragma unroll
    for (int i = 0; i < kBLoads; ++i) store4(f.b[i], b_hi, b_lo, threadIdx.x + i * kThreads);
}

__global__ void __launch_bounds__(kThreads + 32, 1) tf32_gemm_kernel(const __grid_constant__ TfGemmArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ volatile unsigned int s_fail;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    // barriers: full[2] (loaders staged the chunk), empty[2] (its MMAs completed), done, tslot,
    // xbar (the test stall)
    const uint32_t full = base + 2 * kStage, empty = full + 16, done = empty + 16, tslot = done + 8,
                   xbar = done + 16;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));
    const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
    const int n0 = blockIdx.y * kBN;
    const int kb = blockIdx.z * a.kchunk;
    const int ke = min(a.K, kb + a.kchunk);
    const int nk = (ke - kb + kBK - 1) / kBK;

    if (t == 0) {
        s_fail = 0u;
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(full + 8 * i, kThreads);
            tc::mbar_init(empty + 8 * i, 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(xbar, 1);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kBN);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot_ptr;
    const uint32_t cap = tc::cap_polls(a.cap);
    if (tc::stall_requested(a.cap)) {
        // test request: a wait that nothing completes, before any MMA
        if (t == 0 && !tc::mbar_wait_bounded(xbar, 0, cap)) s_fail = 1u;
        __syncthreads();
    }

    if (warp == kThreads / 32) {
        // ---------------- MMA issuer (one lane) ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kBM, kBN);
            for (int c = 0; c < nk; ++c) {
                const int st = c & 1;
                const uint32_t a_hi = base + st * kStage, a_lo = a_hi + kATile, b_hi = a_lo + kATile,
                               b_lo = b_hi + kBTile;
                if (tc::wait_or_fail(&s_fail, full + 8 * st, (c >> 1) & 1u, cap)) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int k = 0; k < kBK / 8; ++k) {
                        const uint64_t ah = tc::smem_desc(a_hi + 32 * k, 1024, tc::SW_128B);
                        const uint64_t al = tc::smem_desc(a_lo + 32 * k, 1024, tc::SW_128B);
                        const uint64_t bh = tc::smem_desc(b_hi + 32 * k, 1024, tc::SW_128B);
                        const uint64_t bl = tc::smem_desc(b_lo + 32 * k, 1024, tc::SW_128B);
                        mma_tf32(tmem, ah, bh, idesc, (c > 0 || k > 0) ? 1u : 0u);
                        mma_tf32(tmem, ah, bl, idesc, 1u);
                        mma_tf32(tmem, al, bh, idesc, 1u);
                    }
                }
                tc::mma_commit(empty + 8 * st);
            }
            tc::mma_commit(done);
        }
    } else {
        // ---------------- loaders: chunk c into stage c & 1, two chunks ahead ----------------
        auto step = [&](int c, Frag &f) {
            const int st = c & 1;
            const uint32_t a_hi = base + st * kStage, a_lo = a_hi + kATile, b_hi = a_lo + kATile,
                           b_lo = b_hi + kBTile;
            // the stage is free once the MMAs of chunk c - 2 have read it
            if (c >= 2) tc::wait_or_fail(&s_fail, empty + 8 * st, ((c - 2) >> 1) & 1u, cap);
            tc::fence_after_sync();
            if (!s_fail) store_frag(f, a_hi, a_lo, b_hi, b_lo);
            if (c + 2 < nk) load_frag(f, a, m0, n0, ke, kb + (c + 2) * kBK);
            tc::fence_proxy_async();
            tc::mbar_arrive(full + 8 * st);
        };
        Frag f0, f1;
        if (nk > 0) load_frag(f0, a, m0, n0, ke, kb);
        if (nk > 1) load_frag(f1, a, m0, n0, ke, kb + kBK);
        for (int c = 0; c < nk; c += 2) {
            step(c, f0);
            if (c + 1 < nk) step(c + 1, f1);
        }
        // every MMA has completed once `done` fires
        tc::wait_or_fail(&s_fail, done, 0u, cap);
        tc::fence_after_sync();
    }
    __syncthreads();  // the operand stages are free for the staged output tile
    if (s_fail) {
        // failure path: `done` tracks every MMA the issuer committed; they
        // must complete before the stages are reused and the TMEM is released
        if (t == kThreads) tc::mbar_wait_bounded(done, 0u, cap);
        __syncthreads();
    }
    tc::fence_after_sync();

    // epilogue (warps 0..7; the issuer warp only passes the barriers).
    // Part 1: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows), columns
    // 32 (w / 4) .. + 31; applies the element-wise step, writes the transposed
    // output (lanes = consecutive rows: coalesced) and stages the tile in
    // shared memory (the operand stages are no longer read).
    const bool worker = warp < kThreads / 32;
    const bool live = __all_sync(0xffffffffu, s_fail == 0u) && nk > 0;  // warp-uniform: tcgen05.ld is collective
    const int q = warp & 3, half = (warp >> 2) & 1;
    const int row = q * 32 + lane;
    const int64_t gr = m0 + row;
    float *sC = reinterpret_cast<float *>(smem_raw + (base - raw));
    const uint32_t taddr = tmem + (static_cast<uint32_t>(q * 32) << 16) + half * 32;
    if (worker) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[16];
            if (live) {
                tc::tmem_ld16(taddr + 16 * h, v);
                tc::tmem_wait_ld();
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = 0.0f;
            }
            const int c0 = half * 32 + 16 * h;
            const bool rok = live && gr < a.M;
            if (a.mode == kTfFwd) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int n = n0 + c0 + e;
                    const float z = v[e] + (n < a.N ? a.bias[n] : 0.0f);
                    v[e] = z;
                    if (rok && n < a.N) a.Ht[static_cast<int64_t>(n) * a.ldt + gr] = silu_f(z);
                }
            } else if (a.mode == kTfBwd) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int n = n0 + c0 + e;
                    const float dz = (rok && n < a.N) ? v[e] * silu_grad_f(a.Zin[gr * a.ldc + n]) : 0.0f;
                    v[e] = dz;
                    if (rok && n < a.N) a.dZt[static_cast<int64_t>(n) * a.ldt + gr] = dz;
                }
            }
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4)
                *reinterpret_cast<float4 *>(sC + row * kCStride + c0 + 4 * e4) =
                    make_float4(v[4 * e4], v[4 * e4 + 1], v[4 * e4 + 2], v[4 * e4 + 3]);
        }
    }
    __syncthreads();
    // part 2: row-major outputs, 16 threads per 64-column row (coalesced)
    for (int i = 0; worker && i < kBM * kBN / 4 / kThreads; ++i) {
        const int idx = t + i * kThreads, r = idx >> 4, c4 = idx & 15;
        const int64_t g = m0 + r;
        const int n = n0 + 4 * c4;
        if (!live || g >= a.M || n >= a.N) continue;
        const float4 v = *reinterpret_cast<const float4 *>(sC + r * kCStride + 4 * c4);
        const float vv[4] = {v.x, v.y, v.z, v.w};
        const bool whole = n + 3 < a.N;
        if (a.mode == kTfFwd) {
            if (whole) {
                *reinterpret_cast<float4 *>(a.Z + g * a.ldc + n) = v;
                *reinterpret_cast<float4 *>(a.H + g * a.ldc + n) =
                    make_float4(silu_f(v.x), silu_f(v.y), silu_f(v.z), silu_f(v.w));
            } else {
                for (int j = 0; j < 4 && n + j < a.N; ++j) {
                    a.Z[g * a.ldc + n + j] = vv[j];
                    a.H[g * a.ldc + n + j] = silu_f(vv[j]);
                }
            }
        } else if (a.mode == kTfBwd) {
            if (whole) *reinterpret_cast<float4 *>(a.dZ + g * a.ldc + n) = v;
            else for (int j = 0; j < 4 && n + j < a.N; ++j) a.dZ[g * a.ldc + n + j] = vv[j];
        } else {
            float *P = a.P + (static_cast<int64_t>(blockIdx.z) * a.M + g) * a.N + n;
            if (whole) *reinterpret_cast<float4 *>(P) = v;
            else for (int j = 0; j < 4 && n + j < a.N; ++j) P[j] = vv[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kBN);
    }
    if (t == 0 && s_fail) atomicExch(a.err, 1u);
}

}  // namespace mtf

size_t tf32_gemm_smem() { return mtf::kSmem; }

cudaError_t tf32_gemm(const TfGemmArgs &a, int slices, cudaStream_t s)
{
    // per device (the current one): set on every launch
    const cudaError_t e = cudaFuncSetAttribute(mtf::tf32_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(mtf::kSmem));
    if (e != cudaSuccess) return e;
    const dim3 grid(static_cast<unsigned>((a.M + mtf::kBM - 1) / mtf::kBM),
                    static_cast<unsigned>((a.N + mtf::kBN - 1) / mtf::kBN), static_cast<unsigned>(slices));
    mtf::tf32_gemm_kernel<<<grid, mtf::kThreads + 32, mtf::kSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbmc
