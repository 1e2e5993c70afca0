// step_f64_aae.cu -- stream-collide kernels of the double storage format, AA even step layout.
#include "step_impl.cuh"

FLB_INSTANTIATE_LAYOUT(double, kAAEven)
