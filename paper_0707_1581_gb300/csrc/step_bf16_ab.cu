// step_bf16_ab.cu -- stream-collide kernels of the __nv_bfloat16 storage format, AB pull layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(__nv_bfloat16, kAB)
