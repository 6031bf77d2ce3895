// 32-byte-lane SpMM kernels: A values E4M3, B F32.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(e4m3, f32, TagE4M3, TagF32)
