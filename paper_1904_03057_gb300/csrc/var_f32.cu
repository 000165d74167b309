// FP32 instantiation of the variable-coefficient operator kernel.
#define BSK_T float
#include "var_impl.cuh"
