// FP32 instantiation: FP32 deviations from w_p n_ref, FP32 arithmetic,
// potential in 64-bit fixed point.
#include "ekl_step.cuh"
EKL_INSTANTIATE(f32, float, float, long long, true)
