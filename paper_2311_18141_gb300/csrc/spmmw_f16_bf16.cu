// 32-byte-lane SpMM kernels: A values F16, B BF16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f16, bf16, TagF16, TagBF16)
