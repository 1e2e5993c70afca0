// step_bf16_aae.cu -- stream-collide kernels of the __nv_bfloat16 storage format, AA even step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(__nv_bfloat16, kAAEven)
