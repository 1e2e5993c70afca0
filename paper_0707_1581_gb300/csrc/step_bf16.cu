// step_bf16.cu -- kernels of the __nv_bfloat16 storage format.
#include "step_impl.cuh"

FLB_INSTANTIATE(__nv_bfloat16)
