// step_f64_aao.cu -- stream-collide kernels of the double storage format, AA odd step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(double, kAAOdd)
