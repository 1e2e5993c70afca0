// step_f32_ab.cu -- stream-collide kernels of the float storage format, AB pull layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(float, kAB)
