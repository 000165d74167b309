// kernels_impl.cuh -- launchers for one element type. Included once by kernels_f32.cu (T=float)
// and once by kernels_f64.cu (T=double) so that the two precisions compile in parallel.
#pragma once

#include "bsk_launch.h"
#include "op_generic.cuh"
#include "vec_kernels.cuh"

namespace bsk {

template <typename T>
static Coef<T> make_coef(const OpLaunch& L)
{
    Coef<T> c;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < kMaxTaps; j++) {
            c.M[d][j] = (T)L.M[d][j];
            c.K[d][j] = (T)L.Kdt[d][j];
        }
    return c;
}

template <typename T, int N, int MODE>
static cudaError_t set_smem_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_op_generic<T, N, MODE, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)generic_smem_bytes<T, N>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_op_generic<T, N, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)generic_smem_bytes<T, N>());
    return e;
}

template <typename T, int N>
static cudaError_t prepare_degree()
{
    cudaError_t e = set_smem_attr<T, N, MODE_OP>();
    if (e == cudaSuccess) e = set_smem_attr<T, N, MODE_MASS>();
    if (e == cudaSuccess) e = set_smem_attr<T, N, MODE_RES>();
    if (e == cudaSuccess) e = set_smem_attr<T, N, MODE_CGP>();
    return e;
}

template <typename T, int N, int MODE>
static cudaError_t launch_generic(const OpLaunch& L, cudaStream_t s)
{
    constexpr size_t smem = generic_smem_bytes<T, N>();
    OpArgs<T> a;
    int tz = 0;
    dim3 grid = op_grid(L.nx, L.ny, L.nz, N, &tz);
    a.g.nx = L.nx;
    a.g.ny = L.ny;
    a.g.nz = L.nz;
    a.g.tz = tz;
    a.g.mask = L.mask;
    a.g.z_off = L.z_off;
    a.g.nz_glob = L.nz_glob > 0 ? L.nz_glob : L.nz;
    a.g.zpad = L.zpad;
    a.c = make_coef<T>(L);
    a.in0 = static_cast<const T*>(L.in0);
    a.in1 = static_cast<const T*>(L.in1);
    a.out0 = static_cast<T*>(L.out0);
    a.out1 = static_cast<T*>(L.out1);
    a.xvec = static_cast<T*>(L.xvec);
    a.b = static_cast<const T*>(L.b);
    a.s = L.s;
    a.sc = L.sc;
    a.partials = L.partials;
    a.fin = L.fin;
    a.p_parity = L.p_parity;
    a.bf16io = L.bf16io;
    a.rb = static_cast<const T*>(L.rb[sizeof(T) == 8]);
    a.jac = MODE == MODE_CGP ? static_cast<const T*>(L.jac[sizeof(T) == 8]) : nullptr;
    a.jn = L.jn;
    a.jvec = MODE == MODE_CGP ? static_cast<const T*>(L.jvec[sizeof(T) == 8]) : nullptr;
    if (a.rb) k_op_generic<T, N, MODE, true><<<grid, kGenNT, smem, s>>>(a);
    else k_op_generic<T, N, MODE, false><<<grid, kGenNT, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t launch_mode(const OpLaunch& L, cudaStream_t s)
{
    switch (L.mode) {
    case MODE_OP: return launch_generic<T, N, MODE_OP>(L, s);
    case MODE_MASS: return launch_generic<T, N, MODE_MASS>(L, s);
    case MODE_RES: return launch_generic<T, N, MODE_RES>(L, s);
    case MODE_CGP: return launch_generic<T, N, MODE_CGP>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_op<BSK_T>(const OpLaunch& L, cudaStream_t s)
{
    if (L.vd[sizeof(BSK_T) == 8] && L.mode != MODE_MASS) return launch_var<BSK_T>(L, s);
    switch (L.degree) {
    case 1: return launch_mode<BSK_T, 1>(L, s);
    case 2: return launch_mode<BSK_T, 2>(L, s);
    case 3: return launch_mode<BSK_T, 3>(L, s);
    case 4: return launch_mode<BSK_T, 4>(L, s);
    case 5: return launch_mode<BSK_T, 5>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t prepare_op<BSK_T>(int degree)
{
    switch (degree) {
    case 1: return prepare_degree<BSK_T, 1>();
    case 2: return prepare_degree<BSK_T, 2>();
    case 3: return prepare_degree<BSK_T, 3>();
    case 4: return prepare_degree<BSK_T, 4>();
    case 5: return prepare_degree<BSK_T, 5>();
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_cg_update<BSK_T>(BSK_T* r, const BSK_T* q, size_t len, Scalars* sc,
                                    double* partials, int fin, cudaStream_t s)
{
    k_cg_update<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(r, q, len, sc, partials, fin);
    return cudaGetLastError();
}

template <>
cudaError_t launch_cg_update_pc<BSK_T>(BSK_T* r, const BSK_T* q, size_t len, int nx, int ny, const BSK_T* jac,
                                       int jn, const BSK_T* jvec, Scalars* sc, double* partials, int fin,
                                       cudaStream_t s)
{
    k_cg_update_pc<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(r, q, len, nx, ny, jac, jn, jvec, sc, partials, fin);
    return cudaGetLastError();
}

template <>
cudaError_t launch_pc_dot<BSK_T>(const BSK_T* r, size_t len, int nx, int ny, const BSK_T* jac, int jn,
                                 const BSK_T* jvec, Scalars* sc, double* partials, cudaStream_t s)
{
    k_pc_dot<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(r, len, nx, ny, jac, jn, jvec, sc, partials);
    return cudaGetLastError();
}

template <>
cudaError_t launch_jacobi_fill<BSK_T>(BSK_T* jinv, size_t len, int nx, int ny, const BSK_T* jac, int jn,
                                      cudaStream_t s)
{
    k_jacobi_fill<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(jinv, len, nx, ny, jac, jn);
    return cudaGetLastError();
}

template <>
cudaError_t launch_cg_flush<BSK_T>(BSK_T* x, const BSK_T* p0, const BSK_T* p1, size_t len,
                                   const Scalars* sc, cudaStream_t s)
{
    k_cg_flush<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(x, p0, p1, len, sc);
    return cudaGetLastError();
}

template <>
cudaError_t launch_cg_init_zero<BSK_T>(const BSK_T* b, BSK_T* r, BSK_T* x, size_t len,
                                       const uint8_t* mask, Scalars* sc, double* partials,
                                       cudaStream_t s)
{
    k_cg_init_zero<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(b, r, x, len, mask, sc, partials);
    return cudaGetLastError();
}

template <>
cudaError_t launch_copy_masked<BSK_T>(const BSK_T* src, BSK_T* dst, size_t len,
                                      const uint8_t* mask, cudaStream_t s)
{
    k_copy_masked<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(src, dst, len, mask);
    return cudaGetLastError();
}

template <>
cudaError_t launch_norm2<BSK_T>(const BSK_T* x, size_t len, Scalars* sc, double* partials,
                                cudaStream_t s)
{
    k_norm2<BSK_T><<<vec_grid(len), kVecNT, 0, s>>>(x, len, sc, partials);
    return cudaGetLastError();
}

}  // namespace bsk
