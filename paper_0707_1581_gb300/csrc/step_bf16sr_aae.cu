// step_bf16sr_aae.cu -- stream-collide kernels of the bf16sr storage format, AA even step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(bf16sr, kAAEven)
