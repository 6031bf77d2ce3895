// Persistent SpMM kernels with B stored as E4M3.
#include "spmm_launch_impl.cuh"

namespace spmm {

cudaError_t launch_spmm_e4m3(int lpn, int vpl, const Problem& p, const LaunchOpts& o,
                           cudaStream_t s) {
    return launch_tag<TagE4M3>(lpn, vpl, p, o, s);
}

}  // namespace spmm
