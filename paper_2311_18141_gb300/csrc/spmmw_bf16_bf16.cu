// 32-byte-lane SpMM kernels: A values BF16, B BF16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(bf16, bf16, TagBF16, TagBF16)
