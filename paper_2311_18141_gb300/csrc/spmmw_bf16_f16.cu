// 32-byte-lane SpMM kernels: A values BF16, B F16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(bf16, f16, TagBF16, TagF16)
