// Persistent SpMM kernels with B stored as F16.
#include "spmm_launch_impl.cuh"

namespace spmm {

cudaError_t launch_spmm_f16(int lpn, int vpl, const Problem& p, const LaunchOpts& o,
                           cudaStream_t s) {
    return launch_tag<TagF16>(lpn, vpl, p, o, s);
}

}  // namespace spmm
