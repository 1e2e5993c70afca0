// step_f64_ab.cu -- stream-collide kernels of the double storage format, AB pull layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(double, kAB)
