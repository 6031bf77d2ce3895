// Launchers of the warp-specialised SpMM kernel (spmm_spec.cuh) for the
// storage pairs it is built for.
#include "launch.cuh"
#include "spmm_spec.cuh"

namespace spmm {

namespace {

template <class TA, class TB, int LPN>
cudaError_t launch_spec_one(const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    using K = KCfg<TA, TB, LPN, 1>;
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    auto kern = spmm_csr_spec<TA, TB, LPN, 1>;
    constexpr int warps = 8;   // four producer/consumer pairs
    const size_t smem = (size_t)spec_smem_bytes(warps, SpecCfg<K>::SLOT_BYTES);
    const int per_sm = cached_ctas_per_sm(kern, warps * 32, smem, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    // units are handed to the producers: half the warps
    const int64_t grid = persistent_grid(per_sm, o.ctas_per_sm, (o.units + K::G - 1) / K::G,
                                         warps / 2);
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(p, o.flags);
    return cudaGetLastError();
}

template <class TA, class TB>
cudaError_t launch_spec(int lpn, const Problem& p, const LaunchOpts& o, cudaStream_t s) {
    switch (lpn) {
        case 8: return launch_spec_one<TA, TB, 8>(p, o, s);
        case 16: return launch_spec_one<TA, TB, 16>(p, o, s);
        case 32: return launch_spec_one<TA, TB, 32>(p, o, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

SpecLaunchFn spec_launcher(int a_dtype, int b_dtype) {
    if (a_dtype == SPMM_F32 && b_dtype == SPMM_F32) return launch_spec<TagF32, TagF32>;
    if (a_dtype == SPMM_F32 && b_dtype == SPMM_BF16) return launch_spec<TagF32, TagBF16>;
    if (a_dtype == SPMM_F16 && b_dtype == SPMM_F32) return launch_spec<TagF16, TagF32>;
    if (a_dtype == SPMM_F16 && b_dtype == SPMM_F16) return launch_spec<TagF16, TagF16>;
    if (a_dtype == SPMM_F16 && b_dtype == SPMM_BF16) return launch_spec<TagF16, TagBF16>;
    return nullptr;
}

}  // namespace spmm
