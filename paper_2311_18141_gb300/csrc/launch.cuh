// Launch helpers for the persistent SpMM kernel instantiations.
#pragma once

#include "common.cuh"

namespace spmm {

struct LaunchOpts {
    int warps_per_cta;   // 4 or 8
    int ctas_per_sm;     // 0 = occupancy limit
    int tile_order;      // steal order
    int64_t units;       // work units (upper bound), caps the grid
};

int device_sm_count();

// Per-B-type dispatchers, one translation unit each (parallel build).
cudaError_t launch_spmm_f32(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s);
cudaError_t launch_spmm_f16(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s);
cudaError_t launch_spmm_bf16(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s);
cudaError_t launch_spmm_e4m3(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s);

}  // namespace spmm
