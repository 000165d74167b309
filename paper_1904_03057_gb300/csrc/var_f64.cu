// FP64 instantiation of the variable-coefficient operator kernel.
#define BSK_T double
#include "var_impl.cuh"
