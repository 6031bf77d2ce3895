// 32-byte-lane SpMM kernels: A values BF16, B E4M3.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(bf16, e4m3, TagBF16, TagE4M3)
