// FP64 instantiation of the operator and vector kernels, plus the precision-conversion kernels
// of the iterative refinement.
#define BSK_T double
#include "kernels_impl.cuh"

namespace bsk {

// Iterative refinement, outer -> inner: r32 = r64 / ||r64|| (||r64||^2 = outer rr_true).
__global__ void __launch_bounds__(kVecNT) k_ir_scale_down(const double* __restrict__ r64,
                                                          float* __restrict__ r32, size_t len,
                                                          const Scalars* outer)
{
    const double inv = 1.0 / sqrt(outer->rr_true);
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        r32[i] = (float)(r64[i] * inv);
}

// Iterative refinement, inner -> outer: x64 += ||r64|| d32.
__global__ void __launch_bounds__(kVecNT) k_ir_update(double* __restrict__ x64,
                                                      const float* __restrict__ d32, size_t len,
                                                      const Scalars* outer)
{
    const double s = sqrt(outer->rr_true);
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        x64[i] = fma(s, (double)d32[i], x64[i]);
}

cudaError_t launch_ir_scale_down(const double* r64, float* r32, size_t len, const Scalars* outer,
                                 cudaStream_t s)
{
    k_ir_scale_down<<<vec_grid(len), kVecNT, 0, s>>>(r64, r32, len, outer);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(double* x64, const float* d32, size_t len, const Scalars* outer,
                             cudaStream_t s)
{
    k_ir_update<<<vec_grid(len), kVecNT, 0, s>>>(x64, d32, len, outer);
    return cudaGetLastError();
}

}  // namespace bsk
