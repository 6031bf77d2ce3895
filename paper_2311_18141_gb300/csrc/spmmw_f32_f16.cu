// 32-byte-lane SpMM kernels: A values F32, B F16.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f32, f16, TagF32, TagF16)
