// step_f32_aae.cu -- stream-collide kernels of the float storage format, AA even step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(float, kAAEven)
