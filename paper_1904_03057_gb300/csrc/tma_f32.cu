// FP32 instantiation of the TMA operator / single-pass CG kernels (degrees 1..5).
#include <cstring>
#define BSK_T float
#define BSK_TMA_HIGH_DEGREE 1
#include "tma_impl.cuh"
