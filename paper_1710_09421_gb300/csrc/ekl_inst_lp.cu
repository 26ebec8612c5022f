// Reduced-precision storage: BF16 or FP16 deviations from w_p n_ref, FP32
// arithmetic, potential in 64-bit fixed point.
#include "ekl_step.cuh"
EKL_INSTANTIATE(bf16, __nv_bfloat16, float, long long, true)
EKL_INSTANTIATE(fp16, __half, float, long long, true)
