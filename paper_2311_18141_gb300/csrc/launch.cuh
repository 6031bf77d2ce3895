// Launch helpers for the persistent SpMM kernel instantiations.
#pragma once

#include <atomic>

#include "common.cuh"

namespace spmm {

struct LaunchOpts {
    int warps_per_cta;   // 1 to 8; 0 = chosen by the launcher
    int ctas_per_sm;     // 0 = occupancy limit
    int flags;           // kFlagOrderColumn | kFlagWarpHome
    int64_t units;       // work units (upper bound), caps the grid
};

int device_sm_count();

// Devices for which per-device launch facts are cached.
constexpr int kMaxDevices = 64;

using LaunchFn = cudaError_t (*)(int lpn, int vpl, const Problem& p, const LaunchOpts& o,
                                 cudaStream_t s);
// 32-byte-lane kernel: lpn lanes per item, nv 32-byte vectors per lane.
using WideLaunchFn = cudaError_t (*)(int lpn, int nv, const Problem& p, const LaunchOpts& o,
                                     cudaStream_t s);

// Warp-specialised kernel: lpn lanes per item, one 16-byte vector per lane.
using SpecLaunchFn = cudaError_t (*)(int lpn, const Problem& p, const LaunchOpts& o,
                                     cudaStream_t s);

struct BatchEntry;
// Batched persistent launch of the products table[0 .. count) of lane shape
// `lpn`: `ctas_per_sm` 0 = occupancy limit.
using BatchLaunchFn = cudaError_t (*)(int lpn, const BatchEntry* table, const int64_t* item_base,
                                      int count, char* ws, int* counter, int64_t max_items,
                                      int ctas_per_sm, cudaStream_t s);

// Resident CTAs per SM of `kern` for `threads` threads and `smem` dynamic
// shared bytes, found once per device, kernel and CTA size (the attribute set
// and the occupancy query stay off the per-call path).  The first query on a
// device raises the kernel's dynamic shared-memory limit to the device's
// opt-in maximum less its static shared memory, so every later launch shape
// fits under it.  0 on a CUDA error.  cache[dev][w - 1] holds CTAs of w warps
// (1 to 8), cache[dev][8] is 1 once the attribute is set.
constexpr int kOccSlots = 9;
template <class Kern>
int cached_ctas_per_sm(Kern kern, int threads, size_t smem,
                       std::atomic<int> (&cache)[kMaxDevices][kOccSlots]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    if (threads < 32 || threads > 256 || threads % 32 != 0) return 0;
    const int slot = threads / 32 - 1;
    int per_sm = cache[dev][slot].load(std::memory_order_relaxed);
    if (per_sm > 0) return per_sm;
    if (cache[dev][kOccSlots - 1].load(std::memory_order_acquire) == 0) {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
            return 0;
        // the limit covers dynamic bytes only: static shared memory counts against it
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        if (dyn_max < 0 || smem > (size_t)dyn_max) return 0;
        if (smem > 0 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) !=
                cudaSuccess)
            return 0;
        if (smem == 0)   // no shared memory: give the SM's whole L1/shared array to L1
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        cache[dev][kOccSlots - 1].store(1, std::memory_order_release);
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
        return 0;
    if (per_sm < 1) per_sm = 1;
    cache[dev][slot].store(per_sm, std::memory_order_relaxed);
    return per_sm;
}

// CTA size of a persistent launch whose tuning leaves it open (0): 7 warps
// when four such CTAs fit on an SM (28 resident warps, the register file and
// the 228 KB of shared memory both just enough at 72 registers and 8 KB of
// staging per warp), else 8 warps.  Found once per device and kernel; 0 on a
// CUDA error.
template <class Kern>
int auto_warps(Kern kern, size_t smem_per_warp,
               std::atomic<int> (&cache)[kMaxDevices][kOccSlots],
               std::atomic<int> (&pick)[kMaxDevices]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    int w = pick[dev].load(std::memory_order_relaxed);
    if (w > 0) return w;
    const int per8 = cached_ctas_per_sm(kern, 256, 8 * smem_per_warp, cache);
    const int per7 = cached_ctas_per_sm(kern, 224, 7 * smem_per_warp, cache);
    if (per8 == 0 || per7 == 0) return 0;
    w = per7 * 7 > per8 * 8 ? 7 : 8;
    pick[dev].store(w, std::memory_order_relaxed);
    return w;
}

// Grid of a persistent launch: SMs x resident CTAs (capped by `ctas_per_sm`
// when given), no more CTAs than there are warp units to hand out.
inline int64_t persistent_grid(int per_sm, int ctas_per_sm, int64_t warp_units, int warps) {
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t grid = (int64_t)device_sm_count() * per_sm;
    const int64_t need = (warp_units + warps - 1) / warps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    return grid;
}

// One launcher per (A value type, B type); one translation unit each so the
// build compiles them in parallel.
#define SPMM_DECLARE_LAUNCHER(a, b)                                                           \
    cudaError_t launch_spmm_##a##_##b(int, int, const Problem&, const LaunchOpts&, cudaStream_t); \
    cudaError_t launch_wide_##a##_##b(int, int, const Problem&, const LaunchOpts&, cudaStream_t); \
    cudaError_t launch_batched_##a##_##b(int, const BatchEntry*, const int64_t*, int, char*,      \
                                         int*, int64_t, int, cudaStream_t);
SPMM_DECLARE_LAUNCHER(f32, f32) SPMM_DECLARE_LAUNCHER(f32, f16)
SPMM_DECLARE_LAUNCHER(f32, bf16) SPMM_DECLARE_LAUNCHER(f32, e4m3)
SPMM_DECLARE_LAUNCHER(f16, f32) SPMM_DECLARE_LAUNCHER(f16, f16)
SPMM_DECLARE_LAUNCHER(f16, bf16) SPMM_DECLARE_LAUNCHER(f16, e4m3)
SPMM_DECLARE_LAUNCHER(bf16, f32) SPMM_DECLARE_LAUNCHER(bf16, f16)
SPMM_DECLARE_LAUNCHER(bf16, bf16) SPMM_DECLARE_LAUNCHER(bf16, e4m3)
SPMM_DECLARE_LAUNCHER(e4m3, f32) SPMM_DECLARE_LAUNCHER(e4m3, f16)
SPMM_DECLARE_LAUNCHER(e4m3, bf16) SPMM_DECLARE_LAUNCHER(e4m3, e4m3)
#undef SPMM_DECLARE_LAUNCHER

// launchers for (a_dtype, b_dtype), both SPMM_F32 .. SPMM_E4M3
LaunchFn spmm_launcher(int a_dtype, int b_dtype);
WideLaunchFn wide_launcher(int a_dtype, int b_dtype);
BatchLaunchFn batched_launcher(int a_dtype, int b_dtype);
// the warp-specialised kernel's launcher, or null for the pairs it is not built for
SpecLaunchFn spec_launcher(int a_dtype, int b_dtype);

}  // namespace spmm
