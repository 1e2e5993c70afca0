// step_f64.cu -- kernels of the double storage format.
#include "step_impl.cuh"

FLB_INSTANTIATE(double)
