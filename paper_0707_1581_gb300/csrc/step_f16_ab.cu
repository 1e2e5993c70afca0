// step_f16_ab.cu -- stream-collide kernels of the __half storage format, AB pull layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(__half, kAB)
