// Persistent SpMM kernels with B stored as F32.
#include "spmm_launch_impl.cuh"

namespace spmm {

cudaError_t launch_spmm_f32(int lpn, int vpl, const Problem& p, const LaunchOpts& o,
                           cudaStream_t s) {
    return launch_tag<TagF32>(lpn, vpl, p, o, s);
}

}  // namespace spmm
