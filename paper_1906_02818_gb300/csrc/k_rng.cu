// The random stream itself (Sec. IV.A: keyed counter-based Philox4x32-10;
// Sec. VI.D: Box-Muller normals), written out by the same device functions
// every path kernel draws from: raw 32-bit words of given blocks of a stream,
// and normals j0 .. j0 + count - 1 of a stream.
#include <cstdint>

#include "mc_kernels.cuh"

namespace gbmc {
namespace {

// Block q0 + i of stream n -> out[4 i .. 4 i + 3] (one 16-byte store per block).
__global__ void __launch_bounds__(256) philox_words_kernel(uint64_t n, uint64_t q0, int64_t blocks,
                                                           uint4 *__restrict__ out,
                                                           const __grid_constant__ RoundKeys rk)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < blocks; i += stride) {
        const uint64_t q = q0 + static_cast<uint64_t>(i);
        if (GBMC_IN_BOUNDS(i, blocks, kDbgPhiloxOut)) out[i] = philox4x32_10(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                          static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32)),
                               rk);
    }
}

// Normals j0 .. j0 + count - 1 of stream n: thread t takes the t-th Philox
// block that overlaps the range and writes the (up to four) normals of it
// that fall inside.
__global__ void __launch_bounds__(256) normals_kernel(uint64_t n, uint64_t j0, int64_t count,
                                                      float *__restrict__ out, const __grid_constant__ RoundKeys rk)
{
    const uint64_t qa = j0 >> 2;
    const int64_t nblk = static_cast<int64_t>(((j0 + static_cast<uint64_t>(count) - 1) >> 2) - qa) + 1;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nblk; i += stride) {
        const uint64_t q = qa + static_cast<uint64_t>(i);
        const float4 z = normals4(q, n, rk);
        const float v[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint64_t j = 4 * q + l;
            if (j >= j0 && j - j0 < static_cast<uint64_t>(count) &&
                GBMC_IN_BOUNDS(static_cast<int64_t>(j - j0), count, kDbgNormalsOut))
                out[j - j0] = v[l];
        }
    }
}

int rng_grid(int64_t work)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    const int64_t need = (work + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    return static_cast<int>(need < cap ? need : cap);
}

}  // namespace
}  // namespace gbmc

extern "C" int mc_philox_words(uint64_t seed, uint64_t stream_index, uint64_t q0, int64_t blocks, uint32_t *dev_out,
                               void *stream)
{
    using namespace gbmc;
    if (!dev_out) return set_last_error(MC_EINVAL, "dev_out is NULL");
    if (reinterpret_cast<uintptr_t>(dev_out) % 16 != 0) return set_last_error(MC_EINVAL, "dev_out must be 16-byte aligned");
    if (blocks < 0 || blocks > (int64_t(1) << 40)) return set_last_error(MC_EINVAL, "blocks outside [0, 2^40]");
    if (blocks > 0 && q0 + static_cast<uint64_t>(blocks - 1) < q0)
        return set_last_error(MC_EINVAL, "block range wraps past 2^64");
    if (blocks == 0) return MC_OK;
    const int grid = rng_grid(blocks);
    if (grid <= 0) return set_last_error(MC_ECUDA, "device query failed");
    const RoundKeys rk = round_keys(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    philox_words_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(stream_index, q0, blocks,
                                                                            reinterpret_cast<uint4 *>(dev_out), rk);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(MC_ECUDA, cudaGetErrorString(e));
    return MC_OK;
}

extern "C" int mc_normals(uint64_t seed, uint64_t stream_index, uint64_t j0, int64_t count, float *dev_out,
                          void *stream)
{
    using namespace gbmc;
    if (!dev_out) return set_last_error(MC_EINVAL, "dev_out is NULL");
    if (count < 0 || count > (int64_t(1) << 40)) return set_last_error(MC_EINVAL, "count outside [0, 2^40]");
    if (count > 0 && j0 + static_cast<uint64_t>(count - 1) < j0)
        return set_last_error(MC_EINVAL, "normal range wraps past 2^64");
    if (count == 0) return MC_OK;
    const int64_t nblk = static_cast<int64_t>(((j0 + static_cast<uint64_t>(count) - 1) >> 2) - (j0 >> 2)) + 1;
    const int grid = rng_grid(nblk);
    if (grid <= 0) return set_last_error(MC_ECUDA, "device query failed");
    const RoundKeys rk = round_keys(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    normals_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(stream_index, j0, count, dev_out, rk);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(MC_ECUDA, cudaGetErrorString(e));
    return MC_OK;
}
