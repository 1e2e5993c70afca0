// step_f16.cu -- kernels of the __half storage format.
#include "step_impl.cuh"

FLB_INSTANTIATE(__half)
