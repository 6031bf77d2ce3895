// 32-byte-lane SpMM kernels: A values F32, B E4M3.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(f32, e4m3, TagF32, TagE4M3)
