// step_f32.cu -- kernels of the float storage format.
#include "step_impl.cuh"

FLB_INSTANTIATE(float)
