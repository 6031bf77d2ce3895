// Launch helpers for the persistent SpMM kernel instantiations.
#pragma once

#include "common.cuh"

namespace spmm {

struct LaunchOpts {
    int warps_per_cta;   // 4 or 8
    int ctas_per_sm;     // 0 = occupancy limit
    int flags;           // kFlagOrderColumn | kFlagWarpHome
    int64_t units;       // work units (upper bound), caps the grid
};

int device_sm_count();

using LaunchFn = cudaError_t (*)(int lpn, int vpl, const Problem& p, const LaunchOpts& o,
                                 cudaStream_t s);

struct BatchEntry;
// Batched persistent launch: `ctas_per_sm` 0 = occupancy limit.
using BatchLaunchFn = cudaError_t (*)(const BatchEntry* table, const int64_t* item_base,
                                      int count, char* ws, int* counter, int64_t max_items,
                                      int ctas_per_sm, cudaStream_t s);

// One launcher per (A value type, B type); one translation unit each so the
// build compiles them in parallel.
#define SPMM_DECLARE_LAUNCHER(a, b)                                                           \
    cudaError_t launch_spmm_##a##_##b(int, int, const Problem&, const LaunchOpts&, cudaStream_t); \
    cudaError_t launch_batched_##a##_##b(const BatchEntry*, const int64_t*, int, char*, int*,     \
                                         int64_t, int, cudaStream_t);
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
BatchLaunchFn batched_launcher(int a_dtype, int b_dtype);

}  // namespace spmm
