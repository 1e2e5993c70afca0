// step_bf16sr_ab.cu -- stream-collide kernels of the bf16sr storage format, AB pull layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(bf16sr, kAB)
