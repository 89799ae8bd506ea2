// BF16 inference of the pricing surrogate on the tensor cores (the network
// of Sec. VI.B evaluated as the DNN-layer analogue of Sec. III.C): one fused
// persistent kernel runs every layer of a 128-row tile with the activations
// in shared memory and the FP32 accumulator in tensor memory.
//
//   layer 0 (n_in -> W):  A0 = [x_hi | x_lo | x_hi] (bf16, K = 32),
//                         B0 = [W0_hi | W0_hi | W0_lo]: x W0 to about
//                         16 bits although both operands are bf16;
//   layers 1..H-1 (W -> W): A = bf16(h), B = bf16(W_l), K = W;
//   epilogues: h = silu(acc + b) in FP32 (silu(v) = v/2 (1 + tanh(v/2)),
//   tanh.approx), rounded to bf16 into the next layer's operand; after the
//   last hidden layer the scalar output y = w_out . h + b_out in FP32.
//
// Warp roles (one CTA of 18 warps per SM; TMEM: 2 x 256 FP32 columns):
//   warp 0   lane 0: TMA producer - streams the pre-swizzled weight chunks
//            (W rows x 32 K columns, 64-byte swizzle) into a ring;
//   warp 1   lane 0: MMA issuer - per layer and tile, K / 16 tcgen05.mma of
//            128 x W x 16 into that tile's accumulator;
//   warps 2..9 / 10..17: epilogue of tile lane X / Y (two tiles in flight,
//            so one tile's epilogue overlaps the other tile's MMAs); thread
//            (warp w, lane l) owns row 32 (w mod 4) + l (its TMEM lane) and
//            half (w - 2 - 8 lane) / 4 of the W columns.
// Every mbarrier wait is bounded; on expiry the CTA stops issuing work and
// writes NaN for the rows it still owes.
#include <cuda_bf16.h>

#include "mc_kernels.cuh"
#include "mlp.cuh"
#include "tc_ptx.cuh"

namespace gbmc {
namespace mlptc {

constexpr int kRows = 128;
constexpr int kKc = 32;                  // K columns per operand panel / weight chunk (64 B rows)
constexpr int kMaxW = 256;
constexpr int kMaxIn = 10;               // 3 n_in <= 32: layer 0 fits one K = 32 panel
constexpr int kMaxLayers = 16;
constexpr int kRing = 5;
static_assert(32 + 16 * kRing + 16 <= 128, "mbarrier words exceed their area");
constexpr int kThreads = 576;
constexpr int kLaneThreads = 256;        // epilogue threads of one tile lane
constexpr int kPanelBytes = kRows * 64;  // one 128 x 32 bf16 panel
constexpr int kSbo = 8 * 64;             // 8-row group stride

struct Args {
    const float *x;        // [n][n_in]
    float *y;              // [n]
    int64_t n;
    int n_in, W, NL;       // NL = hidden layers = MMA layers
    const uint8_t *img;    // weight chunks, W * 64 bytes each
    const float *params;   // packed FP32 parameters (biases, output layer)
    int64_t b_off[kMaxLayers];
    int64_t w_out, b_out;  // offsets of the output layer's weights and bias
    uint32_t cap;
    unsigned int *err;
};

// Byte offset of 16-byte chunk `ch` (0..3) of row `row` in a 64-byte-swizzled
// K-major panel (8-row groups of 512 bytes).
__host__ __device__ constexpr uint32_t sw64(int row, int ch)
{
    return static_cast<uint32_t>((row >> 3) * kSbo + (row & 7) * 64 + ((ch ^ ((row >> 1) & 3)) * 16));
}

__device__ __forceinline__ float tanh_approx(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// silu(v) = v sigmoid(v) = h + h tanh(h), h = v / 2
__device__ __forceinline__ float silu_tanh(float v)
{
    const float h = 0.5f * v;
    return fmaf(h, tanh_approx(h), h);
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void stv4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ void lane_sync(int lane_id)
{
    asm volatile("bar.sync %0, 256;" ::"r"(1 + lane_id) : "memory");
}

// Chunk ids of layer l: 0 for layer 0, else 1 + (l - 1) KC + kc.
__device__ __forceinline__ int chunk_count(int l, int KC) { return l == 0 ? 1 : KC; }
__device__ __forceinline__ int chunk_id(int l, int kc, int KC) { return l == 0 ? 0 : 1 + (l - 1) * KC + kc; }

__global__ void __launch_bounds__(kThreads, 1) mlp_bf16_kernel(const Args a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ float s_part[2][2][kRows];  // [tile lane][column half][row]
    __shared__ volatile unsigned int s_fail;

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int W = a.W, KC = W / kKc, NL = a.NL;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t abytes = static_cast<uint32_t>(KC) * kPanelBytes;  // one tile's activations
    const uint32_t cbytes = static_cast<uint32_t>(W) * 64;            // one weight chunk
    const uint32_t ring = base + 2 * abytes, bars = ring + kRing * cbytes;
    // barrier words: afull[2], dfull[2], lfull[R], lfree[R], tslot, xbar (the
    // failure path's drain of the MMA issuer, and the test stall)
    const uint32_t afull = bars, dfull = bars + 16, lfull = bars + 32, lfree = lfull + 8 * kRing;
    const uint32_t tslot = lfree + 8 * kRing, xbar = tslot + 8;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));

    if (t == 0) {
        s_fail = 0;
        for (int T = 0; T < 2; ++T) {
            tc::mbar_init(afull + 8 * T, kLaneThreads);
            tc::mbar_init(dfull + 8 * T, 1);
        }
        for (int r = 0; r < kRing; ++r) {
            tc::mbar_init(lfull + 8 * r, 1);
            tc::mbar_init(lfree + 8 * r, 1);
        }
        tc::mbar_init(xbar, 1);
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot_ptr;
    const int64_t ntiles = (a.n + kRows - 1) / kRows;
    const int64_t G = gridDim.x;
    const uint32_t cap = tc::cap_polls(a.cap);
    uint32_t issued = 0, lastpar = 0;  // producer: per ring slot, a copy was issued; its lfull parity
    if (tc::stall_requested(a.cap)) {
        // test request: a wait that nothing completes, before any copy or MMA
        if (t == 0 && !tc::mbar_wait_bounded(xbar, 0, cap)) s_fail = 1u;
        __syncthreads();
    }

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t slot = 0, phase = 0, primed = 0;
            for (int64_t tx = blockIdx.x; tx < ntiles; tx += 2 * G) {
                const int lanes = tx + G < ntiles ? 2 : 1;
                for (int l = 0; l < NL; ++l)
                    for (int T = 0; T < lanes; ++T)
                        for (int kc = 0; kc < chunk_count(l, KC); ++kc) {
                            const bool ok = primed < kRing ? (++primed, true)
                                                           : tc::wait_or_fail(&s_fail, lfree + 8 * slot, phase ^ 1u, cap);
                            if (ok && !s_fail) {
                                tc::mbar_arrive_expect_tx(lfull + 8 * slot, cbytes);
                                tc::bulk_g2s(ring + slot * cbytes,
                                             a.img + static_cast<size_t>(chunk_id(l, kc, KC)) * cbytes, cbytes,
                                             lfull + 8 * slot);
                                issued |= 1u << slot;
                                lastpar = (lastpar & ~(1u << slot)) | (phase << slot);
                            }
                            if (++slot == kRing) {
                                slot = 0;
                                phase ^= 1u;
                            }
                        }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kRows, W, true);
            // descriptors change only in their 14-bit start-address field (address / 16)
            const uint64_t adesc0 = tc::smem_desc(base, kSbo, tc::SW_64B);
            const uint64_t bdesc0 = tc::smem_desc(ring, kSbo, tc::SW_64B);
            uint32_t slot = 0, phase = 0, ph[2] = {0, 0};
            for (int64_t tx = blockIdx.x; tx < ntiles; tx += 2 * G) {
                const int lanes = tx + G < ntiles ? 2 : 1;
                for (int l = 0; l < NL; ++l)
                    for (int T = 0; T < lanes; ++T) {
                        const bool aok = tc::wait_or_fail(&s_fail, afull + 8 * T, ph[T], cap);
                        ph[T] ^= 1u;
                        tc::fence_after_sync();
                        for (int kc = 0; kc < chunk_count(l, KC); ++kc) {
                            if (aok && tc::wait_or_fail(&s_fail, lfull + 8 * slot, phase, cap)) {
                                tc::fence_after_sync();
                                const uint64_t ad = adesc0 + ((T * abytes + kc * kPanelBytes) >> 4);
                                const uint64_t bd = bdesc0 + ((slot * cbytes) >> 4);
                                tc::mma_f16(tmem + 256 * T, ad, bd, idesc, kc == 0 ? 0u : 1u);
                                tc::mma_f16(tmem + 256 * T, ad + 2, bd + 2, idesc, 1u);  // K + 16: 32 bytes on
                                tc::mma_commit(lfree + 8 * slot);
                            }
                            if (++slot == kRing) {
                                slot = 0;
                                phase ^= 1u;
                            }
                        }
                        tc::mma_commit(dfull + 8 * T);
                    }
            }
        }
    } else {
        // ---------------- epilogues of tile lane T ----------------
        const int T = (warp - 2) >> 3;
        const int half = ((warp - 2) & 7) >> 2;
        const int row = 32 * (warp & 3) + lane;
        const uint32_t A = base + T * abytes;
        const int ncol = W / 2, col0 = half * ncol;
        const uint32_t taddr = tmem + 256 * T + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + col0;
        uint32_t dph = 0;
        for (int64_t tile = blockIdx.x + T * G; tile < ntiles; tile += 2 * G) {
            const int64_t rg = tile * kRows + row;
            const bool valid = rg < a.n;
            // layer-0 operand, fixed slots: columns 0..9 x_hi, 10..19 x_lo,
            // 20..29 x_hi, 30..31 zero; this thread writes the 16 columns of its half
            if (!s_fail) {
                float hi[kMaxIn], lo[kMaxIn];
#pragma unroll
                for (int k = 0; k < kMaxIn; ++k) {
                    const float xv = (valid && k < a.n_in) ? a.x[rg * a.n_in + k] : 0.0f;
                    hi[k] = __bfloat162float(__float2bfloat16_rn(xv));
                    lo[k] = xv - hi[k];
                }
                float col[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) col[j] = j < 10 ? hi[j] : j < 20 ? lo[j - 10] : j < 30 ? hi[j - 20] : 0.0f;
                uint32_t w8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    w8[e] = half ? bf2(col[16 + 2 * e], col[17 + 2 * e]) : bf2(col[2 * e], col[2 * e + 1]);
                stv4(A + sw64(row, 2 * half), w8[0], w8[1], w8[2], w8[3]);
                stv4(A + sw64(row, 2 * half + 1), w8[4], w8[5], w8[6], w8[7]);
                tc::fence_proxy_async();
            }
            tc::fence_before_sync();
            tc::mbar_arrive(afull + 8 * T);
            for (int l = 0; l < NL; ++l) {
                tc::wait_or_fail(&s_fail, dfull + 8 * T, dph, cap);
                dph ^= 1u;
                tc::fence_after_sync();
                const bool live = __all_sync(0xffffffffu, s_fail == 0u);
                const bool last = l == NL - 1;
                const float *bias = a.params + a.b_off[l];
                float acc_out = 0.0f;
                for (int cc = 0; cc < ncol; cc += 16) {
                    float v[16];
                    if (live) {
                        tc::tmem_ld16(taddr + cc, v);
                        tc::tmem_wait_ld();
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] = 0.0f;
                    }
                    const int c = col0 + cc;
#pragma unroll
                    for (int e4 = 0; e4 < 4; ++e4) {
                        const float4 b4 = __ldg(reinterpret_cast<const float4 *>(bias + c) + e4);
                        v[4 * e4] = silu_tanh(v[4 * e4] + b4.x);
                        v[4 * e4 + 1] = silu_tanh(v[4 * e4 + 1] + b4.y);
                        v[4 * e4 + 2] = silu_tanh(v[4 * e4 + 2] + b4.z);
                        v[4 * e4 + 3] = silu_tanh(v[4 * e4 + 3] + b4.w);
                    }
                    if (!last) {
                        const uint32_t pan = A + (c / kKc) * kPanelBytes;
                        const int ch = (c % kKc) / 8;
                        stv4(pan + sw64(row, ch), bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
                        stv4(pan + sw64(row, ch + 1), bf2(v[8], v[9]), bf2(v[10], v[11]), bf2(v[12], v[13]),
                             bf2(v[14], v[15]));
                    } else {
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4) {
                            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(a.params + a.w_out + c) + e4);
                            acc_out = fmaf(w4.x, v[4 * e4], acc_out);
                            acc_out = fmaf(w4.y, v[4 * e4 + 1], acc_out);
                            acc_out = fmaf(w4.z, v[4 * e4 + 2], acc_out);
                            acc_out = fmaf(w4.w, v[4 * e4 + 3], acc_out);
                        }
                    }
                }
                if (!last) {
                    tc::fence_proxy_async();
                    tc::fence_before_sync();
                    tc::mbar_arrive(afull + 8 * T);
                } else {
                    s_part[T][half][row] = acc_out;
                    lane_sync(T);
                    if (half == 0 && valid) {
                        const float yv = s_part[T][0][row] + s_part[T][1][row] + __ldg(a.params + a.b_out);
                        if (GBMC_IN_BOUNDS(rg, a.n, kDbgMlpOut)) a.y[rg] = live ? yv : __int_as_float(0x7fc00000);
                    }
                    lane_sync(T);  // s_part is reused by the next tile
                }
            }
        }
    }
    __syncthreads();
    if (s_fail) {
        // failure path, before the shared memory and TMEM are released: the
        // producer waits for the last copy into each ring slot, and one more
        // commit of the MMA issuer tracks every MMA it issued (xbar is still
        // in phase 0: waiting never completes a phase)
        if (t == 0)
            for (int r = 0; r < kRing; ++r)
                if ((issued >> r) & 1u) tc::mbar_wait_bounded(lfull + 8 * r, (lastpar >> r) & 1u, cap);
        if (t == 32) {
            tc::mma_commit(xbar);
            tc::mbar_wait_bounded(xbar, 0u, cap);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
    if (t == 0 && s_fail) atomicExch(a.err, 1u);
}

struct Offsets {
    int64_t w[kMaxLayers + 1];
};

// Weight image: chunk 0 = layer 0 (per output unit: columns 0..9 W0_hi,
// 10..19 W0_hi, 20..29 W0_lo over the inputs, zero past n_in), chunk
// 1 + (l - 1) KC + kc = columns 32 kc .. 32 kc + 31 of W_l^T; each chunk W
// rows x 64 bytes in the 64-byte-swizzled K-major layout.
__global__ void mlp_bf16_prep_kernel(int n_in, int W, int NL, const float *params, const Offsets off, uint8_t *img)
{
    const int KC = W / kKc;
    const int64_t nchunks = 1 + static_cast<int64_t>(NL - 1) * KC;
    const int64_t total = nchunks * W * kKc;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(i % kKc);
        const int nrow = static_cast<int>((i / kKc) % W);
        const int64_t cid = i / (static_cast<int64_t>(kKc) * W);
        float v = 0.0f;
        if (cid == 0) {
            const int kin = k % 10;
            if (k < 30 && kin < n_in) {
                const float w = params[off.w[0] + static_cast<int64_t>(kin) * W + nrow];  // W0 [n_in][W]
                const float hi = __bfloat162float(__float2bfloat16_rn(w));
                v = k < 20 ? hi : w - hi;
            }
        } else {
            const int64_t l = 1 + (cid - 1) / KC, kc = (cid - 1) % KC;
            v = params[off.w[l] + (kc * kKc + k) * W + nrow];  // W_l [W][W]: in x out
        }
        const uint32_t o = sw64(nrow, k / 8) + (k % 8) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(img + cid * W * 64 + o) = __float2bfloat16_rn(v);
    }
}

}  // namespace mlptc

bool mlp_bf16_supported(const MlpLayout &L)
{
    const int n_in = L.sizes.front(), hidden = static_cast<int>(L.sizes.size()) - 2;
    if (n_in < 1 || n_in > mlptc::kMaxIn || hidden < 1 || hidden > mlptc::kMaxLayers) return false;
    const int W = L.sizes[1];
    if (W % mlptc::kKc != 0 || W > mlptc::kMaxW) return false;
    for (int l = 1; l <= hidden; ++l)
        if (L.sizes[l] != W) return false;
    return L.sizes.back() == 1;
}

size_t mlp_bf16_image_bytes(const MlpLayout &L)
{
    const int W = L.sizes[1], hidden = static_cast<int>(L.sizes.size()) - 2;
    return static_cast<size_t>(1 + (hidden - 1) * (W / mlptc::kKc)) * W * 64;
}

cudaError_t mlp_bf16_prepare(const MlpLayout &L, const float *params, uint8_t *img, cudaStream_t s)
{
    const int hidden = static_cast<int>(L.sizes.size()) - 2;
    mlptc::Offsets off{};
    for (int l = 0; l < hidden; ++l) off.w[l] = L.w_off[l];
    mlptc::mlp_bf16_prep_kernel<<<256, 256, 0, s>>>(L.sizes[0], L.sizes[1], hidden, params, off, img);
    return cudaGetLastError();
}

cudaError_t mlp_forward_bf16(const MlpLayout &L, const float *params, const uint8_t *img, const float *x, int64_t n,
                             float *y, unsigned int *err, uint32_t cap, cudaStream_t s)
{
    using namespace mlptc;
    Args a{};
    a.x = x;
    a.y = y;
    a.n = n;
    a.n_in = L.sizes[0];
    a.W = L.sizes[1];
    a.NL = static_cast<int>(L.sizes.size()) - 2;
    a.img = img;
    a.params = params;
    for (int l = 0; l < a.NL; ++l) a.b_off[l] = L.b_off[l];
    a.w_out = L.w_off[a.NL];
    a.b_out = L.b_off[a.NL];
    a.cap = cap;
    a.err = err;
    const int KC = a.W / kKc;
    // at least half the SM's shared memory: one CTA per SM, which owns all 512 TMEM columns
    int smem = 1024 + 2 * KC * kPanelBytes + kRing * a.W * 64 + 128;  // barriers: 16 + 16 + 16 R + 8 + 8 <= 128
    if (smem < 120 * 1024) smem = 120 * 1024;
    cudaError_t e = cudaFuncSetAttribute(mlp_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t ntiles = (n + kRows - 1) / kRows;
    const int64_t pairs = (ntiles + 1) / 2;
    const int grid = static_cast<int>(pairs < sms ? pairs : sms);
    mlp_bf16_kernel<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbmc
