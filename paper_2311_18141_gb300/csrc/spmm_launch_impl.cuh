// Instantiates the persistent SpMM kernels for one (A value type, B type).
#pragma once

#include "batch_kernel.cuh"
#include "launch.cuh"
#include "spmm_kernel.cuh"
#include "spmm_wide.cuh"

namespace spmm {

template <class TA, class TB, int LPN, int VPL>
cudaError_t launch_one(const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    static std::atomic<int> pick[kMaxDevices];
    auto kern = spmm_csr_persistent<TA, TB, LPN, VPL>;
    constexpr int stage = KCfg<TA, TB, LPN, VPL>::STAGE_BYTES;
    const int warps = o.warps_per_cta > 0 ? o.warps_per_cta : auto_warps(kern, stage, cache, pick);
    if (warps == 0) return cudaErrorInvalidValue;
    const int threads = warps * 32;
    const size_t smem = (size_t)smem_bytes(warps, stage);
    const int per_sm = cached_ctas_per_sm(kern, threads, smem, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    // o.units counts plan chunks; a warp's unit is G of them
    constexpr int G = KCfg<TA, TB, LPN, VPL>::G;
    const int64_t grid = persistent_grid(per_sm, o.ctas_per_sm, (o.units + G - 1) / G, warps);
    kern<<<(unsigned)grid, threads, smem, s>>>(p, o.flags);
    return cudaGetLastError();
}

template <class TA, class TB, int LPN, int NV>
cudaError_t launch_wide_one(const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    auto kern = spmm_csr_wide<TA, TB, LPN, NV>;
    const int threads = (o.warps_per_cta > 0 ? o.warps_per_cta : 8) * 32;
    const int per_sm = cached_ctas_per_sm(kern, threads, 0, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    constexpr int G = WCfg<TA, TB, LPN, NV>::G;
    const int64_t grid = persistent_grid(per_sm, o.ctas_per_sm, (o.units + G - 1) / G,
                                         threads / 32);
    kern<<<(unsigned)grid, threads, 0, s>>>(p, o.flags);
    return cudaGetLastError();
}

template <class TA, class TB>
cudaError_t launch_pair(int lpn, int vpl, const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    switch (lpn * 10 + vpl) {
        case 21: return launch_one<TA, TB, 2, 1>(p, o, s);
        case 24: return launch_one<TA, TB, 2, 4>(p, o, s);
        case 41: return launch_one<TA, TB, 4, 1>(p, o, s);
        case 42: return launch_one<TA, TB, 4, 2>(p, o, s);
        case 81: return launch_one<TA, TB, 8, 1>(p, o, s);
        case 161: return launch_one<TA, TB, 16, 1>(p, o, s);
        case 321: return launch_one<TA, TB, 32, 1>(p, o, s);
        case 322: return launch_one<TA, TB, 32, 2>(p, o, s);
        case 324: return launch_one<TA, TB, 32, 4>(p, o, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class TA, class TB>
cudaError_t launch_wide_pair(int lpn, int nv, const Problem& p, const LaunchOpts& o,
                             cudaStream_t s) {
    if (nv != 1) return cudaErrorInvalidValue;
    switch (lpn) {
        case 2: return launch_wide_one<TA, TB, 2, 1>(p, o, s);
        case 4: return launch_wide_one<TA, TB, 4, 1>(p, o, s);
        case 8: return launch_wide_one<TA, TB, 8, 1>(p, o, s);
        case 16: return launch_wide_one<TA, TB, 16, 1>(p, o, s);
        case 32: return launch_wide_one<TA, TB, 32, 1>(p, o, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class TA, class TB, int LPN>
cudaError_t launch_batched_one(const BatchEntry* table, const int64_t* item_base, int count,
                               char* ws, int* counter, int64_t max_items, int ctas_per_sm,
                               cudaStream_t s) {
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    auto kern = spmm_csr_batched_kernel<TA, TB, LPN>;
    const int threads = kBatchWarps * 32;
    const size_t smem = (size_t)smem_bytes(kBatchWarps, batch_stage_bytes<TA, TB, LPN>());
    const int per_sm = cached_ctas_per_sm(kern, threads, smem, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    const int64_t grid = persistent_grid(per_sm, ctas_per_sm, max_items, kBatchWarps);
    kern<<<(unsigned)grid, threads, smem, s>>>(table, item_base, count, ws, counter);
    return cudaGetLastError();
}

template <class TA, class TB>
cudaError_t launch_batched(int lpn, const BatchEntry* table, const int64_t* item_base, int count,
                           char* ws, int* counter, int64_t max_items, int ctas_per_sm,
                           cudaStream_t s) {
    switch (lpn) {
        case 2: return launch_batched_one<TA, TB, 2>(table, item_base, count, ws, counter,
                                                     max_items, ctas_per_sm, s);
        case 4: return launch_batched_one<TA, TB, 4>(table, item_base, count, ws, counter,
                                                     max_items, ctas_per_sm, s);
        case 8: return launch_batched_one<TA, TB, 8>(table, item_base, count, ws, counter,
                                                     max_items, ctas_per_sm, s);
        case 16: return launch_batched_one<TA, TB, 16>(table, item_base, count, ws, counter,
                                                       max_items, ctas_per_sm, s);
        case 32: return launch_batched_one<TA, TB, 32>(table, item_base, count, ws, counter,
                                                       max_items, ctas_per_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spmm

// The staged and batched kernels of one (A, B) pair, and its 32-byte-lane
// kernels: separate translation units so that the build compiles them in
// parallel.
#define SPMM_DEFINE_LAUNCHER(a, b, TA, TB)                                               \
    namespace spmm {                                                                      \
    cudaError_t launch_spmm_##a##_##b(int lpn, int vpl, const Problem& p,                \
                                      const LaunchOpts& o, cudaStream_t s) {              \
        return launch_pair<TA, TB>(lpn, vpl, p, o, s);                                    \
    }                                                                                     \
    cudaError_t launch_batched_##a##_##b(int lpn, const BatchEntry* t, const int64_t* ib, \
                                         int n, char* ws, int* ctr, int64_t mx, int cps,  \
                                         cudaStream_t s) {                                \
        return launch_batched<TA, TB>(lpn, t, ib, n, ws, ctr, mx, cps, s);                \
    }                                                                                     \
    }

#define SPMM_DEFINE_WIDE_LAUNCHER(a, b, TA, TB)                                          \
    namespace spmm {                                                                      \
    cudaError_t launch_wide_##a##_##b(int lpn, int nv, const Problem& p,                 \
                                      const LaunchOpts& o, cudaStream_t s) {              \
        return launch_wide_pair<TA, TB>(lpn, nv, p, o, s);                                \
    }                                                                                     \
    }
