// FP64 instantiation of the TMA operator / single-pass CG kernels (degrees 1..3; higher degrees
// exceed the shared-memory budget in FP64 and use the general kernel).
#include <cstring>
#define BSK_T double
#define BSK_TMA_HIGH_DEGREE 0
#include "tma_impl.cuh"
