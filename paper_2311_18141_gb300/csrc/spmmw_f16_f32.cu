// 32-byte-lane SpMM kernels: A values F16, B F32.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f16, f32, TagF16, TagF32)
