// transform.cu -- banded line solves and transfers: the direct B-spline transform at the grid
// nodes, and the coarse-to-fine prolongation of Robin problems. The direct transform (section 2.3 and Fig.
// figBspnSignProc of arXiv:1904.03057: interpolation, samples f -> coefficients c). Along one
// axis the sampled odd-reflected basis B (B[j][i] = psi_i(x_j)) is a symmetric positive
// definite band matrix of half-width p = ceil((n + 1) / 2) - 1, so c = (Bz^-1 (x) By^-1 (x)
// Bx^-1) f is three passes of banded triangular solves, one thread per grid line, with the
// Cholesky factor of B computed once on the host. The indirect transform (c -> u at the nodes)
// is the separable convolution with the sampled B-spline and runs on the operator kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bsk_launch.h"

namespace bsk {

namespace {

constexpr int kSolveNT = 128;

// L: N rows of (P + 1) entries, row j = { 1 / L[j][j], L[j][j-1], ..., L[j][j-P] } (entries that
// would reach before row 0 are zero). One thread per grid line along `axis`.
template <typename T, int P>
__global__ void __launch_bounds__(kSolveNT) k_band_solve(T* __restrict__ d, int nx, int ny, int nz, int axis,
                                                         const T* __restrict__ L)
{
    const long long line = blockIdx.x * (long long)kSolveNT + threadIdx.x;
    int N;
    size_t base, stride;
    if (axis == 0) {          // x lines, one per (z, y)
        if (line >= (long long)ny * nz) return;
        N = nx; stride = 1; base = (size_t)line * nx;
    } else if (axis == 1) {   // y lines, one per (z, x)
        if (line >= (long long)nx * nz) return;
        const long long z = line / nx, x = line % nx;
        N = ny; stride = (size_t)nx; base = (size_t)z * ny * nx + (size_t)x;
    } else {                  // z lines, one per (y, x)
        if (line >= (long long)nx * ny) return;
        N = nz; stride = (size_t)nx * ny; base = (size_t)line;
    }
    constexpr int w = P + 1;
    // forward: y_j = (f_j - sum_k L[j][j-k] y_{j-k}) / L[j][j]; prev[k-1] = y_{j-k}
    T prev[P > 0 ? P : 1];
#pragma unroll
    for (int k = 0; k < P; k++) prev[k] = T(0);
    for (int j = 0; j < N; j++) {
        const T* Lj = L + (size_t)j * w;
        T v = d[base + (size_t)j * stride];
#pragma unroll
        for (int k = 1; k <= P; k++) v -= Lj[k] * prev[k - 1];
        v *= Lj[0];
        d[base + (size_t)j * stride] = v;
#pragma unroll
        for (int k = P - 1; k > 0; k--) prev[k] = prev[k - 1];
        if (P > 0) prev[0] = v;
    }
    // backward: c_j = (y_j - sum_k L[j+k][j] c_{j+k}) / L[j][j]; prev[k-1] = c_{j+k}
#pragma unroll
    for (int k = 0; k < P; k++) prev[k] = T(0);
    for (int j = N - 1; j >= 0; j--) {
        T v = d[base + (size_t)j * stride];
#pragma unroll
        for (int k = 1; k <= P; k++)
            if (j + k < N) v -= L[(size_t)(j + k) * w + k] * prev[k - 1];
        v *= L[(size_t)j * w];
        d[base + (size_t)j * stride] = v;
#pragma unroll
        for (int k = P - 1; k > 0; k--) prev[k] = prev[k - 1];
        if (P > 0) prev[0] = v;
    }
}

// out[.., f, ..] = sum_{k < w} tab[f * w + k] in[.., c0[f] + k, ..] along `axis` (rows of a banded
// rectangular matrix; columns outside the input are skipped). One thread per output element.
template <typename T>
__global__ void __launch_bounds__(256) k_transfer(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                  int nz, int axis, int nout, int w, const T* __restrict__ tab,
                                                  const int* __restrict__ c0)
{
    const int ox = axis == 0 ? nout : nx, oy = axis == 1 ? nout : ny, oz = axis == 2 ? nout : nz;
    const size_t total = (size_t)ox * oy * oz;
    const int nin = axis == 0 ? nx : axis == 1 ? ny : nz;
    const size_t stride = axis == 0 ? 1 : axis == 1 ? (size_t)nx : (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % ox);
        const int y = (int)((i / ox) % oy);
        const int z = (int)(i / ((size_t)ox * oy));
        const int f = axis == 0 ? x : axis == 1 ? y : z;
        size_t ib = ((size_t)(axis == 2 ? 0 : z) * ny + (axis == 1 ? 0 : y)) * nx + (axis == 0 ? 0 : x);
        T acc = T(0);
        const int c = c0[f];
        for (int k = 0; k < w; k++) {
            const int cc = c + k;
            if (cc >= 0 && cc < nin) acc = fma(tab[(size_t)f * w + k], in[ib + (size_t)cc * stride], acc);
        }
        out[i] = acc;
    }
}

template <typename S, typename D>
__global__ void __launch_bounds__(256) k_convert(const S* __restrict__ src, D* __restrict__ dst, size_t len)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

}  // namespace

cudaError_t launch_convert_f32_f64(const float* src, double* dst, size_t len, cudaStream_t s)
{
    k_convert<float, double><<<vec_grid(len), 256, 0, s>>>(src, dst, len);
    return cudaGetLastError();
}

cudaError_t launch_convert_f64_f32(const double* src, float* dst, size_t len, cudaStream_t s)
{
    k_convert<double, float><<<vec_grid(len), 256, 0, s>>>(src, dst, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve(T* d, int nx, int ny, int nz, int axis, int p, const T* L, cudaStream_t s)
{
    const long long lines = axis == 0 ? (long long)ny * nz : axis == 1 ? (long long)nx * nz : (long long)nx * ny;
    const unsigned blocks = (unsigned)((lines + kSolveNT - 1) / kSolveNT);
    switch (p) {
    case 0: k_band_solve<T, 0><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    case 1: k_band_solve<T, 1><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    case 2: k_band_solve<T, 2><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    case 3: k_band_solve<T, 3><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    case 4: k_band_solve<T, 4><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    case 5: k_band_solve<T, 5><<<blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, L); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transfer(const T* in, T* out, int nx, int ny, int nz, int axis, int nout, int w,
                            const T* tab, const int* c0, cudaStream_t s)
{
    const size_t total = (size_t)(axis == 0 ? nout : nx) * (axis == 1 ? nout : ny) * (axis == 2 ? nout : nz);
    const size_t blocks = std::min<size_t>((total + 255) / 256, (size_t)152 * 16);
    k_transfer<T><<<(unsigned)std::max<size_t>(blocks, 1), 256, 0, s>>>(in, out, nx, ny, nz, axis, nout, w, tab, c0);
    return cudaGetLastError();
}

template cudaError_t launch_band_solve<float>(float*, int, int, int, int, int, const float*, cudaStream_t);
template cudaError_t launch_band_solve<double>(double*, int, int, int, int, int, const double*, cudaStream_t);
template cudaError_t launch_transfer<float>(const float*, float*, int, int, int, int, int, int, const float*,
                                            const int*, cudaStream_t);
template cudaError_t launch_transfer<double>(const double*, double*, int, int, int, int, int, int, const double*,
                                             const int*, cudaStream_t);

}  // namespace bsk
