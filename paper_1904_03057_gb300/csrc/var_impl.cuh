// var_impl.cuh -- host side of the variable-coefficient operator kernel (op_var.cuh) for one
// element type: Gauss-point tables, grid, launch. Included once by var_f32.cu (T = float) and
// once by var_f64.cu (T = double).
#pragma once

#include <cmath>

#include "bsk_launch.h"
#include "host_bspline.h"
#include "op_var.cuh"

namespace bsk {
namespace {

// Tables of one cell: local coordinate xi in [0, 1] of a knot interval; the cell's n + 1
// B-splines are centred at offsets lo + t (lo = -floor(n/2)) from the interval's reference
// node, and the interval starts at offset 0 (odd n, integer knots) or -1/2 (even n).
template <typename T>
VarTabs<T> make_tabs(int n, const double h[3])
{
    VarTabs<T> tb{};
    double xi[kVarMaxQ], w[kVarMaxQ];
    const int q = (3 * n + 2) / 2, lo = -(n / 2);
    const double o = (n & 1) ? 0.0 : -0.5;
    host::gauss_unit(q, xi, w);
    for (int g = 0; g < q; g++) {
        tb.w[g] = (T)w[g];
        for (int t = 0; t <= n; t++) {
            const double u = o + xi[g] - lo - t;
            const double b = host::bspline(n, u), du = host::bspline_deriv(n, u);
            tb.B[g][t] = (T)b;
            for (int ax = 0; ax < 3; ax++) tb.D[ax][g][t] = (T)(du / h[ax]);
            tb.Bw[g][t] = (T)(w[g] * b);
            tb.Dxw[g][t] = (T)(w[g] * du / h[0]);
        }
    }
    return tb;
}

template <typename T, int N, int MODE>
cudaError_t set_var_attr()
{
    return cudaFuncSetAttribute(k_op_var<T, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)VarCfg<T, N>::smem);
}

template <typename T, int N>
cudaError_t prepare_var_degree()
{
    cudaError_t e = set_var_attr<T, N, MODE_OP>();
    if (e == cudaSuccess) e = set_var_attr<T, N, MODE_RES>();
    if (e == cudaSuccess) e = set_var_attr<T, N, MODE_CGP>();
    return e;
}

template <typename T, int N>
dim3 var_grid_n(int nx, int ny, int nz, int* tz)
{
    constexpr int TT = VarCfg<T, N>::TT;
    const int bx = (nx + TT - 1) / TT, by = (ny + TT - 1) / TT;
    const long long bxy = (long long)bx * by;
    // about four blocks per SM, but at least 2n output planes per block so that the n extra
    // z-cells each block recomputes stay a bounded overhead
    const long long nzc = (608 + bxy - 1) / bxy;
    int t = (int)((nz + nzc - 1) / nzc);
    if (t < 2 * N) t = 2 * N;
    if (t > nz) t = nz;
    *tz = t;
    return dim3(bx, by, (nz + t - 1) / t);
}

template <typename T>
dim3 var_grid_t(int degree, int nx, int ny, int nz, int* tz)
{
    switch (degree) {
    case 1: return var_grid_n<T, 1>(nx, ny, nz, tz);
    case 2: return var_grid_n<T, 2>(nx, ny, nz, tz);
    case 3: return var_grid_n<T, 3>(nx, ny, nz, tz);
    case 4: return var_grid_n<T, 4>(nx, ny, nz, tz);
    default: return var_grid_n<T, 5>(nx, ny, nz, tz);
    }
}

template <typename T, int N, int MODE>
cudaError_t launch_var_mode(const OpLaunch& L, cudaStream_t s)
{
    using Cfg = VarCfg<T, N>;
    VarArgs<T> a;
    int tz = 0;
    const dim3 grid = var_grid_n<T, N>(L.nx, L.ny, L.nz, &tz);
    a.g.nx = L.nx;
    a.g.ny = L.ny;
    a.g.nz = L.nz;
    a.g.tz = tz;
    a.g.mask = L.mask;
    a.t = make_tabs<T>(N, L.h);
    a.vol = (T)(L.h[0] * L.h[1] * L.h[2]);
    a.dt = (T)L.dt;
    a.d = static_cast<const T*>(L.vd[sizeof(T) == 8]);
    a.m = static_cast<const T*>(L.vm[sizeof(T) == 8]);
    a.in0 = static_cast<const T*>(L.in0);
    a.in1 = static_cast<const T*>(L.in1);
    a.out0 = static_cast<T*>(L.out0);
    a.out1 = static_cast<T*>(L.out1);
    a.xvec = static_cast<T*>(L.xvec);
    a.b = static_cast<const T*>(L.b);
    a.jvec = MODE == MODE_CGP ? static_cast<const T*>(L.jvec[sizeof(T) == 8]) : nullptr;
    a.sc = L.sc;
    a.partials = L.partials;
    a.fin = L.fin;
    a.p_parity = L.p_parity;
    k_op_var<T, N, MODE><<<grid, Cfg::NT, Cfg::smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_var_n(const OpLaunch& L, cudaStream_t s)
{
    switch (L.mode) {
    case MODE_OP: return launch_var_mode<T, N, MODE_OP>(L, s);
    case MODE_RES: return launch_var_mode<T, N, MODE_RES>(L, s);
    case MODE_CGP: return launch_var_mode<T, N, MODE_CGP>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_coef_fill(const double* __restrict__ src, BSK_T* __restrict__ dst, size_t len)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src ? (BSK_T)src[i] : BSK_T(1);
}

// Probing the diagonal of a banded operator: nodes whose coordinates equal (cx, cy, cz) modulo
// `stride` (n + 1) are more than n apart on some axis, as are their mirror images, so one
// application of A to their indicator vector returns A_ll at each of them.
__global__ void k_probe_fill(BSK_T* __restrict__ v, int nx, int ny, size_t len, int stride, int cx, int cy,
                             int cz, const uint8_t* __restrict__ mask)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const bool on = x % stride == cx && y % stride == cy && z % stride == cz && (!mask || mask[i]);
        v[i] = on ? BSK_T(1) : BSK_T(0);
    }
}

// jinv[i] = 1 / y[i] at the probed nodes; after every colour, every active node holds 1 / A_ii
// (inactive nodes get 1: their residual is zero).
__global__ void k_probe_take(const BSK_T* __restrict__ y, BSK_T* __restrict__ jinv, int nx, int ny, size_t len,
                             int stride, int cx, int cy, int cz, const uint8_t* __restrict__ mask)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y2 = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        if (x % stride == cx && y2 % stride == cy && z % stride == cz)
            jinv[i] = (!mask || mask[i]) ? BSK_T(1) / y[i] : BSK_T(1);
    }
}

}  // namespace

template <>
cudaError_t launch_probe<BSK_T>(BSK_T* v, const BSK_T* y, BSK_T* jinv, int take, int nx, int ny, int nz,
                                int stride, int cx, int cy, int cz, const uint8_t* mask, cudaStream_t s)
{
    const size_t len = (size_t)nx * ny * nz;
    if (take) k_probe_take<<<vec_grid(len), 256, 0, s>>>(y, jinv, nx, ny, len, stride, cx, cy, cz, mask);
    else k_probe_fill<<<vec_grid(len), 256, 0, s>>>(v, nx, ny, len, stride, cx, cy, cz, mask);
    return cudaGetLastError();
}

template <>
cudaError_t launch_coef_fill<BSK_T>(const double* src, BSK_T* dst, size_t len, cudaStream_t s)
{
    k_coef_fill<<<vec_grid(len), 256, 0, s>>>(src, dst, len);
    return cudaGetLastError();
}

template <>
cudaError_t launch_var<BSK_T>(const OpLaunch& L, cudaStream_t s)
{
    switch (L.degree) {
    case 1: return launch_var_n<BSK_T, 1>(L, s);
    case 2: return launch_var_n<BSK_T, 2>(L, s);
    case 3: return launch_var_n<BSK_T, 3>(L, s);
    case 4: return launch_var_n<BSK_T, 4>(L, s);
    case 5: return launch_var_n<BSK_T, 5>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t prepare_var<BSK_T>(int degree)
{
    switch (degree) {
    case 1: return prepare_var_degree<BSK_T, 1>();
    case 2: return prepare_var_degree<BSK_T, 2>();
    case 3: return prepare_var_degree<BSK_T, 3>();
    case 4: return prepare_var_degree<BSK_T, 4>();
    case 5: return prepare_var_degree<BSK_T, 5>();
    default: return cudaErrorInvalidValue;
    }
}

template <>
size_t var_grid_blocks<BSK_T>(int nx, int ny, int nz, int degree)
{
    int tz = 0;
    const dim3 g = var_grid_t<BSK_T>(degree, nx, ny, nz, &tz);
    return (size_t)g.x * g.y * g.z;
}

template <>
double var_flops_per_node<BSK_T>(int degree, int nx, int ny, int nz)
{
    // floating-point operations the kernel executes per output node (FMA = 2), counting the
    // recomputed halo cells of each block: z-pass 4(n+1) FMA per halo node and quad plane;
    // BC 5(n+1) FMA (+ 2 products with folded weights) per y-pass node, 10(n+1) FMA + 4 (folded)
    // or 8 products per x quad point;
    // DE 3 Q (n+1) FMA per output column and quad plane plus 2(n+1) per z-transpose.
    const int n = degree, q = (3 * n + 2) / 2, nb = n + 1;
    const double ny_prod = n <= 3 ? 2 : 0, pt_prod = n <= 3 ? 4 : 8;   // VarCfg::FOLD
    int tile = 0;
    switch (degree) {
    case 1: tile = VarCfg<BSK_T, 1>::TT; break;
    case 2: tile = VarCfg<BSK_T, 2>::TT; break;
    case 3: tile = VarCfg<BSK_T, 3>::TT; break;
    case 4: tile = VarCfg<BSK_T, 4>::TT; break;
    default: tile = VarCfg<BSK_T, 5>::TT; break;
    }
    const double H = tile + 2 * n, C = tile + n, QC = q * C;
    const double per_cell = 2.0 * (q * H * H * 4 * nb)                        // A
                            + q * QC * H * (2.0 * 5 * nb + ny_prod)            // BC y-pass
                            + q * QC * C * q * (2.0 * 10 * nb + pt_prod)       // BC x-pass
                            + 2.0 * tile * tile * q * (3.0 * q * nb + 2 * nb); // DE
    int tz = 0;
    const dim3 g = var_grid_t<BSK_T>(degree, nx, ny, nz, &tz);
    const double cells = (double)g.x * g.y * ((double)nz + (double)g.z * n);
    return per_cell * cells / ((double)nx * ny * nz);
}

}  // namespace bsk
