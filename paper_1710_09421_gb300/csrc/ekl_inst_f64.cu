// FP64 instantiation: FP64 populations and arithmetic, FP64 potential.
// Compiled with -fmad=false so that every product and sum rounds on its own,
// as in a plain CPU evaluation of the same formulas.
#include "ekl_step.cuh"
EKL_INSTANTIATE(f64, double, double, double, false)
