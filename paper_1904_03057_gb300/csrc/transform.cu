// transform.cu -- the direct B-spline transform at the grid nodes (section 2.3 and Fig.
// figBspnSignProc of arXiv:1904.03057: interpolation, samples f -> coefficients c). Along one
// axis the sampled odd-reflected basis B (B[j][i] = psi_i(x_j)) is a symmetric positive
// definite band matrix of half-width p = ceil((n + 1) / 2) - 1, so c = (Bz^-1 (x) By^-1 (x)
// Bx^-1) f is three passes of banded triangular solves, one thread per grid line, with the
// Cholesky factor of B computed once on the host. The indirect transform (c -> u at the nodes)
// is the separable convolution with the sampled B-spline and runs on the operator kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsk_launch.h"

namespace bsk {

namespace {

constexpr int kSolveNT = 128;

// L: N rows of (p + 1) entries, row j = { 1 / L[j][j], L[j][j-1], ..., L[j][j-p] }.
template <typename T>
__global__ void __launch_bounds__(kSolveNT) k_band_solve(T* __restrict__ d, int nx, int ny, int nz, int axis, int p,
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
    const int w = p + 1;
    // forward: y_j = (f_j - sum_k L[j][j-k] y_{j-k}) / L[j][j]
    T y1 = T(0), y2 = T(0);   // y_{j-1}, y_{j-2}
    for (int j = 0; j < N; j++) {
        const T* Lj = L + (size_t)j * w;
        T v = d[base + (size_t)j * stride];
        if (p >= 1) v -= Lj[1] * y1;
        if (p >= 2) v -= Lj[2] * y2;
        v *= Lj[0];
        d[base + (size_t)j * stride] = v;
        y2 = y1;
        y1 = v;
    }
    // backward: c_j = (y_j - sum_k L[j+k][j] c_{j+k}) / L[j][j]
    T c1 = T(0), c2 = T(0);   // c_{j+1}, c_{j+2}
    for (int j = N - 1; j >= 0; j--) {
        T v = d[base + (size_t)j * stride];
        if (p >= 1 && j + 1 < N) v -= L[(size_t)(j + 1) * w + 1] * c1;
        if (p >= 2 && j + 2 < N) v -= L[(size_t)(j + 2) * w + 2] * c2;
        v *= L[(size_t)j * w];
        d[base + (size_t)j * stride] = v;
        c2 = c1;
        c1 = v;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_band_solve(T* d, int nx, int ny, int nz, int axis, int p, const T* L, cudaStream_t s)
{
    const long long lines = axis == 0 ? (long long)ny * nz : axis == 1 ? (long long)nx * nz : (long long)nx * ny;
    const long long blocks = (lines + kSolveNT - 1) / kSolveNT;
    k_band_solve<T><<<(unsigned)blocks, kSolveNT, 0, s>>>(d, nx, ny, nz, axis, p, L);
    return cudaGetLastError();
}

template cudaError_t launch_band_solve<float>(float*, int, int, int, int, int, const float*, cudaStream_t);
template cudaError_t launch_band_solve<double>(double*, int, int, int, int, int, const double*, cudaStream_t);

}  // namespace bsk
