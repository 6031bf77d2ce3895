// 32-byte-lane SpMM kernels: A values F32, B BF16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f32, bf16, TagF32, TagBF16)
