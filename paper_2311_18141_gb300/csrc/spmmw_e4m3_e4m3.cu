// 32-byte-lane SpMM kernels: A values E4M3, B E4M3.
#include "spmm_launch_impl.cuh"

SPMM_DEFINE_WIDE_LAUNCHER(e4m3, e4m3, TagE4M3, TagE4M3)
