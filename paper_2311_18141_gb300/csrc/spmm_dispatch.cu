// Table of persistent-kernel launchers indexed by (A value type, B type).
#include "launch.cuh"

namespace spmm {

LaunchFn spmm_launcher(int a_dtype, int b_dtype) {
    static const LaunchFn table[4][4] = {
        {launch_spmm_f32_f32, launch_spmm_f32_f16, launch_spmm_f32_bf16, launch_spmm_f32_e4m3},
        {launch_spmm_f16_f32, launch_spmm_f16_f16, launch_spmm_f16_bf16, launch_spmm_f16_e4m3},
        {launch_spmm_bf16_f32, launch_spmm_bf16_f16, launch_spmm_bf16_bf16, launch_spmm_bf16_e4m3},
        {launch_spmm_e4m3_f32, launch_spmm_e4m3_f16, launch_spmm_e4m3_bf16, launch_spmm_e4m3_e4m3},
    };
    if (a_dtype < 0 || a_dtype > 3 || b_dtype < 0 || b_dtype > 3) return nullptr;
    return table[a_dtype][b_dtype];
}

WideLaunchFn wide_launcher(int a_dtype, int b_dtype) {
    static const WideLaunchFn table[4][4] = {
        {launch_wide_f32_f32, launch_wide_f32_f16, launch_wide_f32_bf16, launch_wide_f32_e4m3},
        {launch_wide_f16_f32, launch_wide_f16_f16, launch_wide_f16_bf16, launch_wide_f16_e4m3},
        {launch_wide_bf16_f32, launch_wide_bf16_f16, launch_wide_bf16_bf16, launch_wide_bf16_e4m3},
        {launch_wide_e4m3_f32, launch_wide_e4m3_f16, launch_wide_e4m3_bf16, launch_wide_e4m3_e4m3},
    };
    if (a_dtype < 0 || a_dtype > 3 || b_dtype < 0 || b_dtype > 3) return nullptr;
    return table[a_dtype][b_dtype];
}

BatchLaunchFn batched_launcher(int a_dtype, int b_dtype) {
    static const BatchLaunchFn table[4][4] = {
        {launch_batched_f32_f32, launch_batched_f32_f16, launch_batched_f32_bf16,
         launch_batched_f32_e4m3},
        {launch_batched_f16_f32, launch_batched_f16_f16, launch_batched_f16_bf16,
         launch_batched_f16_e4m3},
        {launch_batched_bf16_f32, launch_batched_bf16_f16, launch_batched_bf16_bf16,
         launch_batched_bf16_e4m3},
        {launch_batched_e4m3_f32, launch_batched_e4m3_f16, launch_batched_e4m3_bf16,
         launch_batched_e4m3_e4m3},
    };
    if (a_dtype < 0 || a_dtype > 3 || b_dtype < 0 || b_dtype > 3) return nullptr;
    return table[a_dtype][b_dtype];
}

}  // namespace spmm
