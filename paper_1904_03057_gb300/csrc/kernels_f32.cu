// FP32 instantiation of the operator and vector kernels.
#define BSK_T float
#include "kernels_impl.cuh"
