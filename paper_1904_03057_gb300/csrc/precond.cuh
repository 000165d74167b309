// precond.cuh -- the reciprocal of the Jacobi preconditioner (op_generic.cuh, vec_kernels.cuh).
#pragma once

#include <cuda_runtime.h>

namespace bsk {

// 1 / d for the Jacobi preconditioner. FP32: the division. FP64: the FP32 reciprocal refined by
// one step of Newton's iteration for 1/d, r <- r (2 - d r), which squares the relative error
// (about 2^-24 -> 2^-48) for a few FP64 multiply-adds instead of a division on the FP64 pipe
// (1/62 of the FP32 rate on GB300); values outside the float range take the division.
__device__ __forceinline__ float recip_pc(float d) { return 1.0f / d; }
__device__ __forceinline__ double recip_pc(double d)
{
    const float f = (float)d;
    const float r0 = __frcp_rn(f);
    if (!(fabsf(f) >= 1e-36f && fabsf(f) <= 1e36f)) return 1.0 / d;
    double r = (double)r0;
    r = r * fma(-d, r, 2.0);
    return r;
}

}  // namespace bsk
