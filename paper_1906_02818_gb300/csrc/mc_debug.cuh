// Bounds checks of the debug build (compiled with GBMC_DEBUG; nothing in the
// release build).  A kernel's access whose index falls outside its buffer is
// skipped and recorded: the first failure's site code and index, and a
// count, in this translation unit's device words; nothing traps, so the
// kernel and the context carry on.  mc_debug_status reads and clears the
// words of every translation unit (each registers a reader at load time).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbmc {

// Site codes (mc_debug_status reports the first failing one).
enum DebugSite : unsigned {
    kDbgGbm1dSave = 1, kDbgBasketSave = 2, kDbgHestonSave = 3, kDbgCkptStore = 4, kDbgCkptLoad = 5,
    kDbgMlpOut = 6, kDbgPhiloxOut = 7, kDbgNormalsOut = 8, kDbgLabelOut = 9
};

// Registry of the translation units' readers (mc_api.cu): a reader copies
// and clears its unit's words.
using DebugReader = int (*)(unsigned long long *first, unsigned *count);
void debug_register(DebugReader fn);

#ifdef GBMC_DEBUG
namespace {
__device__ unsigned long long g_dbg_first;  // (code << 48) | (index mod 2^48); 0 = none
__device__ unsigned int g_dbg_count;

__device__ __forceinline__ bool dbg_in_bounds(int64_t idx, int64_t len, unsigned code)
{
    if (idx >= 0 && idx < len) return true;
    atomicCAS(&g_dbg_first, 0ull,
              (static_cast<unsigned long long>(code) << 48) | (static_cast<unsigned long long>(idx) & 0xFFFFFFFFFFFFull));
    atomicAdd(&g_dbg_count, 1u);
    return false;
}

int dbg_read_unit(unsigned long long *first, unsigned *count)
{
    const unsigned long long z = 0;
    const unsigned zc = 0;
    if (cudaMemcpyFromSymbol(first, g_dbg_first, sizeof *first) != cudaSuccess ||
        cudaMemcpyFromSymbol(count, g_dbg_count, sizeof *count) != cudaSuccess ||
        cudaMemcpyToSymbol(g_dbg_first, &z, sizeof z) != cudaSuccess ||
        cudaMemcpyToSymbol(g_dbg_count, &zc, sizeof zc) != cudaSuccess)
        return -1;
    return 0;
}

struct DbgRegistrar {
    DbgRegistrar() { debug_register(&dbg_read_unit); }
} g_dbg_registrar;
}  // namespace
#define GBMC_IN_BOUNDS(idx, len, code) ::gbmc::dbg_in_bounds((idx), (len), (code))
#else
#define GBMC_IN_BOUNDS(idx, len, code) true
#endif

}  // namespace gbmc
