// Instantiates the persistent SpMM kernel for one (A value type, B type).
#pragma once

#include "batch_kernel.cuh"
#include "launch.cuh"
#include "spmm_kernel.cuh"

namespace spmm {

template <class TA, class TB, int LPN, int VPL>
cudaError_t launch_one(const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    auto kern = spmm_csr_persistent<TA, TB, LPN, VPL>;
    const int threads = o.warps_per_cta * 32;
    const size_t smem = (size_t)smem_bytes(o.warps_per_cta, KCfg<TA, TB, LPN, VPL>::STAGE_BYTES);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int64_t grid = (int64_t)device_sm_count() * per_sm;
    // o.units counts plan chunks; a warp's unit is G of them
    constexpr int G = KCfg<TA, TB, LPN, VPL>::G;
    const int64_t warp_units = (o.units + G - 1) / G;
    const int64_t need = (warp_units + o.warps_per_cta - 1) / o.warps_per_cta;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, s>>>(p, o.flags);
    return cudaGetLastError();
}

template <class TA, class TB>
cudaError_t launch_pair(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    switch (lpn * 10 + vpl) {
        case 21: return launch_one<TA, TB, 2, 1>(p, o, s);
        case 41: return launch_one<TA, TB, 4, 1>(p, o, s);
        case 81: return launch_one<TA, TB, 8, 1>(p, o, s);
        case 161: return launch_one<TA, TB, 16, 1>(p, o, s);
        case 321: return launch_one<TA, TB, 32, 1>(p, o, s);
        case 322: return launch_one<TA, TB, 32, 2>(p, o, s);
        case 324: return launch_one<TA, TB, 32, 4>(p, o, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class TA, class TB>
cudaError_t launch_batched(const BatchEntry* table, const int64_t* item_base, int count, char* ws,
                           int* counter, int64_t max_items, int ctas_per_sm, cudaStream_t s) {
    auto kern = spmm_csr_batched_kernel<TA, TB>;
    const int threads = kBatchWarps * 32;
    const size_t smem = (size_t)smem_bytes(kBatchWarps, batch_stage_bytes<TA, TB>());
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t grid = (int64_t)device_sm_count() * per_sm;
    const int64_t need = (max_items + kBatchWarps - 1) / kBatchWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, s>>>(table, item_base, count, ws, counter);
    return cudaGetLastError();
}

}  // namespace spmm

#define SPMM_DEFINE_LAUNCHER(a, b, TA, TB)                                               \
    namespace spmm {                                                                      \
    cudaError_t launch_spmm_##a##_##b(int lpn, int vpl, const Problem& p,                \
                                      const LaunchOpts& o, cudaStream_t s) {              \
        return launch_pair<TA, TB>(lpn, vpl, p, o, s);                                    \
    }                                                                                     \
    cudaError_t launch_batched_##a##_##b(const BatchEntry* t, const int64_t* ib, int n,  \
                                         char* ws, int* ctr, int64_t mx, int cps,         \
                                         cudaStream_t s) {                                \
        return launch_batched<TA, TB>(t, ib, n, ws, ctr, mx, cps, s);                     \
    }                                                                                     \
    }
