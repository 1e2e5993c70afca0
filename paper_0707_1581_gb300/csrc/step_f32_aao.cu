// step_f32_aao.cu -- stream-collide kernels of the float storage format, AA odd step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(float, kAAOdd)
