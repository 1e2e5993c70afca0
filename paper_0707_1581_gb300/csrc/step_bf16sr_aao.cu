// step_bf16sr_aao.cu -- stream-collide kernels of the bf16sr storage format, AA odd step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(bf16sr, kAAOdd)
