// vec_kernels.cuh -- streaming CG vector kernels (section 2.5 of arXiv:1904.03057) with fused
// FP64 reductions.
#pragma once

#include "bsk_device.cuh"

namespace bsk {

constexpr int kVecNT = 256;

// r -= alpha q; reduction r.r; finaliser `fin` (FIN_UPD in a solve: beta, convergence).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_cg_update(T* __restrict__ r, const T* __restrict__ q,
                                                      size_t len, Scalars* sc, double* partials,
                                                      int fin)
{
    if (*(volatile int*)&sc->done) return;
    const T alpha = (T)sc->alpha;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = fma(-alpha, q[i], r[i]);
        r[i] = v;
        acc += (double)v * (double)v;
    }
    grid_reduce2<kVecNT>(acc, 0.0, partials, sc, fin, 0);
}

// x += alpha_prev p[p_cur]: applies the last deferred update once the iteration has stopped.
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_cg_flush(T* __restrict__ x, const T* __restrict__ p0,
                                                     const T* __restrict__ p1, size_t len,
                                                     const Scalars* sc)
{
    const T ap = (T)sc->alpha_prev;
    const T* p = sc->p_cur ? p1 : p0;
    if (ap == T(0)) return;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        x[i] = fma(ap, p[i], x[i]);
}

// CG start from x = 0: r = mask(b), x = 0; reduction r.r = b.b; finaliser FIN_RES_INIT.
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_cg_init_zero(const T* __restrict__ b, T* __restrict__ r,
                                                         T* __restrict__ x, size_t len,
                                                         const uint8_t* __restrict__ mask,
                                                         Scalars* sc, double* partials)
{
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = (!mask || mask[i]) ? b[i] : T(0);
        r[i] = v;
        x[i] = T(0);
        acc += (double)v * (double)v;
    }
    grid_reduce2<kVecNT>(acc, acc, partials, sc, FIN_RES_INIT, 0);
}

// dst = mask ? src : 0 (src == dst allowed)
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_copy_masked(const T* src, T* dst, size_t len,
                                                        const uint8_t* __restrict__ mask)
{
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        dst[i] = (!mask || mask[i]) ? src[i] : T(0);
}

// reduction x.x; finaliser FIN_NORM (rr_true).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_norm2(const T* __restrict__ x, size_t len, Scalars* sc,
                                                  double* partials)
{
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        acc += (double)x[i] * (double)x[i];
    grid_reduce2<kVecNT>(acc, 0.0, partials, sc, FIN_NORM, 0);
}

}  // namespace bsk
