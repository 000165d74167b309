// vec_kernels.cuh -- streaming CG vector kernels (section 2.5 of arXiv:1904.03057) with fused
// reductions (FP64 across threads and blocks), including the Jacobi-preconditioned variants
// (the solver of the large run of section 3).
#pragma once

#include "bsk_device.cuh"
#include "precond.cuh"

namespace bsk {

constexpr int kVecNT = 256;

// Per-thread sum of squares: compensated FP32 for float vectors (GB300 runs FP64 at 1/62 of
// the FP32 rate, so FP64 per-element arithmetic would dominate these streaming kernels), plain
// FP64 for double vectors; widened to FP64 once per thread for the deterministic reduction.
template <typename T>
struct SqSum {
    double s = 0.0;
    __device__ __forceinline__ void add(T v) { s = fma((double)v, (double)v, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SqSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = __fsub_rn(__fmul_rn(v, v), c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// r -= alpha q; reduction r.r; finaliser `fin` (FIN_UPD in a solve: beta, convergence).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_cg_update(T* __restrict__ r, const T* __restrict__ q,
                                                      size_t len, Scalars* sc, double* partials,
                                                      int fin)
{
    if (*(volatile int*)&sc->done) return;
    const T alpha = (T)sc->alpha;
    SqSum<T> acc;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = fma(-alpha, q[i], r[i]);
        r[i] = v;
        acc.add(v);
    }
    grid_reduce2<kVecNT>(acc.value(), 0.0, partials, sc, fin, 0);
}

// Compensated running sum of arbitrary terms: Kahan in FP32 for float kernels, plain FP64 for
// double kernels (widened once per thread for the grid reduction).
template <typename T>
struct TermSum {
    double s = 0.0;
    __device__ __forceinline__ void add(T v) { s += (double)v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct TermSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Jacobi factors of flat index i of an nx * ny * nz grid (op_generic.cuh, jacobi_inv).
template <typename T>
__device__ __forceinline__ T jacobi_inv_flat(const T* jac, int jn, size_t i, int nx, int ny)
{
    const size_t xy = (size_t)nx * ny;
    const int z = (int)(i / xy);
    const size_t rem = i - (size_t)z * xy;
    const int y = (int)(rem / nx), x = (int)(rem - (size_t)y * nx);
    const T mx = jac[x], kx = jac[jn + x], my = jac[2 * jn + y], ky = jac[3 * jn + y];
    const T mz = jac[4 * jn + z], kz = jac[5 * jn + z];
    return recip_pc(mz * my * (mx + kx) + (kz * my + mz * ky) * mx);
}

// Preconditioned CG residual pass: r -= alpha q; reductions r.r (convergence) and r.z with
// z = r / diag A (Jacobi); finaliser FIN_UPD_PC.
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_cg_update_pc(T* __restrict__ r, const T* __restrict__ q,
                                                         size_t len, int nx, int ny, const T* __restrict__ jac,
                                                         int jn, const T* __restrict__ jvec, Scalars* sc,
                                                         double* partials, int fin)
{
    if (*(volatile int*)&sc->done) return;
    const T alpha = (T)sc->alpha;
    SqSum<T> rr;
    TermSum<T> rz;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = fma(-alpha, q[i], r[i]);
        r[i] = v;
        rr.add(v);
        rz.add(v * v * (jvec ? jvec[i] : jacobi_inv_flat(jac, jn, i, nx, ny)));
    }
    grid_reduce2<kVecNT>(rr.value(), rz.value(), partials, sc, fin, 0);
}

// r.z with z = r / diag A: the starting value of the preconditioned iteration (FIN_PC_INIT).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_pc_dot(const T* __restrict__ r, size_t len, int nx, int ny,
                                                   const T* __restrict__ jac, int jn, const T* __restrict__ jvec,
                                                   Scalars* sc, double* partials)
{
    TermSum<T> rz;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = r[i];
        rz.add(v * v * (jvec ? jvec[i] : jacobi_inv_flat(jac, jn, i, nx, ny)));
    }
    grid_reduce2<kVecNT>(rz.value(), 0.0, partials, sc, FIN_PC_INIT, 0);
}

// jinv[i] = 1 / diag A at flat index i: the per-node vector the preconditioned passes read, so
// that the diagonal is formed once per solve setting rather than at every use (in FP64 on GB300
// the formation costs more than the 8 bytes per node of the read).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_jacobi_fill(T* __restrict__ jinv, size_t len, int nx, int ny,
                                                        const T* __restrict__ jac, int jn)
{
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        jinv[i] = jacobi_inv_flat(jac, jn, i, nx, ny);
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
    SqSum<T> acc;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT) {
        const T v = (!mask || mask[i]) ? b[i] : T(0);
        r[i] = v;
        x[i] = T(0);
        acc.add(v);
    }
    grid_reduce2<kVecNT>(acc.value(), acc.value(), partials, sc, FIN_RES_INIT, 0);
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

// reduction x.x; finaliser FIN_NORM (rr_true). Not on a solver path: FP64 per element, so the
// result is a reference value for checks (bsk_norm2).
template <typename T>
__global__ void __launch_bounds__(kVecNT) k_norm2(const T* __restrict__ x, size_t len, Scalars* sc,
                                                  double* partials)
{
    SqSum<double> acc;
    for (size_t i = blockIdx.x * (size_t)kVecNT + threadIdx.x; i < len;
         i += (size_t)gridDim.x * kVecNT)
        acc.add(x[i]);
    grid_reduce2<kVecNT>(acc.value(), 0.0, partials, sc, FIN_NORM, 0);
}

}  // namespace bsk
