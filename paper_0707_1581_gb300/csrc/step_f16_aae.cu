// step_f16_aae.cu -- stream-collide kernels of the __half storage format, AA even step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(__half, kAAEven)
