// Double-float instantiation of the TMA kernel: y = A x and r = b - A x with FP64 inputs and
// outputs and the operator evaluated in double-float arithmetic on the FP32 pipes (degrees
// 1..3; no CG passes).
#include <cstring>

#include "dfloat.cuh"
#define BSK_T bsk::dfl
#define BSK_TMA_HIGH_DEGREE 0
#define BSK_TMA_NO_CG 1
#include "tma_impl.cuh"
