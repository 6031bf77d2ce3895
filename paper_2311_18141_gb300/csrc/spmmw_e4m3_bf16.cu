// 32-byte-lane SpMM kernels: A values E4M3, B BF16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(e4m3, bf16, TagE4M3, TagBF16)
