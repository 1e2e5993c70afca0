// step_bf16sr.cu -- kernels of the bfloat16 format with stochastic rounding.
#include "step_impl.cuh"

FLB_INSTANTIATE(bf16sr)
