// step_f16_aao.cu -- stream-collide kernels of the __half storage format, AA odd step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(__half, kAAOdd)
