// 32-byte-lane SpMM kernels: A values F16, B E4M3.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f16, e4m3, TagF16, TagE4M3)
