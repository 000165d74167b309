// op_generic.cuh -- fused three-sweep operator kernel, general layout (any grid size, any
// degree 1..5, FP32 or FP64).
//
// One block owns a 32 x 16 (x, y) output tile and marches along z over `tz` planes. Per output
// plane it stages one new masked, odd-reflected input plane (tile + halo n on each side) into a
// ring of 2n+1 planes in shared memory, then runs the three 1-D sweeps of Fig. FiltAlg
// (arXiv:1904.03057, section 2.4) back to back on shared memory:
//   z-sweep on the halo tile    P = Mz x,          Q = dt Kz x
//   y-sweep on the x-halo tile  A = My P,          S = A + dt Ky P + My Q
//   x-sweep on the output tile  y = Mx S + dt Kx A
// which is M M M x + dt (K M M + M K M + M M K) x with 7 band convolutions per point (the
// mass-only variant runs 3). Depending on the mode the kernel also fuses the CG vector work of
// section 2.5 around the operator: the search-direction update p = r + beta p_old on the fly
// while staging (p = r / diag A + beta p_old with the Jacobi preconditioner of the large run of
// section 3), the deferred x update, the residual b - A x, and the p.Ap / r.r reductions.
// The RB instantiation takes Robin (boundary penalty) problems: the untruncated basis with zero
// ghosts, and the band rows of the n + 1 positions nearest each face read from a table (the
// integrals there are truncated to the box and carry the penalty term).
#pragma once

#include <cuda_bf16.h>

#include "bsk_device.cuh"
#include "precond.cuh"

namespace bsk {

template <typename T>
struct OpArgs {
    Geom g;
    Coef<T> c;
    const T* in0;     // x (OP, RES), r (CGP), u (MASS)
    const T* in1;     // p_old (CGP), q (MASS, may be null)
    T* out0;          // y (OP, MASS), r (RES), q = A p (CGP)
    T* out1;          // p (CGP)
    T* xvec;          // x, updated in place (CGP)
    const T* b;       // right-hand side (RES)
    double s;         // MASS: weight of in1
    Scalars* sc;
    double* partials;
    int fin;
    int p_parity;
    int bf16io;       // FP32, OP / MASS: in0, in1 and out0 are bfloat16 arrays (BF16 storage)
    const T* rb;      // Robin problems: band rows near the faces (robin_row), null otherwise
    const T* jac;     // CGP: Jacobi diagonal factors (jacobi_inv), null = no preconditioner
    int jn;           // row length of jac
    const T* jvec;    // CGP: 1 / diag A per node (Jacobi), read instead of forming it from jac
};

// Robin (boundary penalty) problems use the untruncated basis with integrals truncated to the
// box, so the 1-D band matrices differ from the shift-invariant kernels in the first and last
// N + 1 rows of each axis. rb holds those rows: [2 (mass, stiffness + penalty)][3 axes][2 ends]
// [N + 1 rows][2N + 1 taps], the stiffness rows already weighted by dt and including the face
// term penalty * (beta_a beta_b at the face). Returns the row of axis ax at position pos, or null
// where the shift-invariant taps apply (and for positions outside the grid).
template <typename T, int N>
__device__ __forceinline__ const T* robin_row(const T* rb, int m, int ax, int pos, int len)
{
    constexpr int NR = N + 1, W = 2 * N + 1;
    int end, row;
    if (pos < NR) {
        end = 0;
        row = pos;
    } else if (pos >= len - NR && pos < len) {
        end = 1;
        row = pos - (len - NR);
    } else {
        return nullptr;
    }
    return rb + ((((size_t)m * 3 + ax) * 2 + end) * NR + row) * W;
}

// 1 / diag(A) at node (x, y, z) from the per-axis diagonals of the band matrices:
// jac = [3 axes][2 (mass, stiffness incl. dt and penalty)][jn], so that
// diag = mz my mx + kz my mx + mz ky mx + mz my kx (the diagonal of the separable operator).
template <typename T>
__device__ __forceinline__ T jacobi_inv(const T* j, int jn, int x, int y, int z)
{
    const T mx = j[x], kx = j[jn + x], my = j[2 * jn + y], ky = j[3 * jn + y];
    const T mz = j[4 * jn + z], kz = j[5 * jn + z];
    return recip_pc(mz * my * (mx + kx) + (kz * my + mz * ky) * mx);
}

// Element o of an input / output array that holds T, or bfloat16 when bf (FP32 kernels only).
template <typename T>
__device__ __forceinline__ T ld_io(const T* p, size_t o, int bf)
{
    if constexpr (sizeof(T) == 4) {
        if (bf) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[o]);
    }
    return p[o];
}
template <typename T>
__device__ __forceinline__ void st_io(T* p, size_t o, T v, int bf)
{
    if constexpr (sizeof(T) == 4) {
        if (bf) {
            reinterpret_cast<__nv_bfloat16*>(p)[o] = __float2bfloat16_rn(v);
            return;
        }
    }
    p[o] = v;
}

template <typename T, int N>
constexpr size_t generic_smem_bytes()
{
    constexpr int L = 2 * N + 1, HX = kGenTX + 2 * N, HY = kGenTY + 2 * N;
    return sizeof(T) * (size_t)(L * HY * HX + 2 * HY * HX + 2 * kGenTY * HX);
}

template <typename T, int N, int MODE, bool RB>
__global__ void __launch_bounds__(kGenNT) k_op_generic(const __grid_constant__ OpArgs<T> a)
{
    constexpr int L = 2 * N + 1;
    constexpr int TX = kGenTX, TY = kGenTY, NT = kGenNT;
    constexpr int HX = TX + 2 * N, HY = TY + 2 * N;
    constexpr bool MASS_ONLY = (MODE == MODE_MASS);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* sP = ring + L * HY * HX;
    T* sQ = sP + HY * HX;
    T* sA = sQ + HY * HX;
    T* sS = sA + TY * HX;

    const int tid = threadIdx.x;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const uint8_t* __restrict__ mask = a.g.mask;

    T beta = T(0), alpha_prev = T(0);
    if (MODE == MODE_CGP) {
        if (*(volatile int*)&a.sc->done) return;  // uniform over the grid
        beta = (T)a.sc->beta;
        alpha_prev = (T)a.sc->alpha_prev;
    }

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.g.tz;
    const int z1 = min(z0 + a.g.tz, nz);
    const int zbase = z0 - N;

    auto load_plane = [&](int gz) {
        T* dst = ring + ((gz - zbase) % L) * (HY * HX);
        int sz = 0;
        int sgz;
        if (RB) {
            sz = gz;
            sgz = (unsigned)gz < (unsigned)nz;
        } else {
            // local plane gz is global plane z_off + gz (a whole grid: z_off = 0, no padding)
            sgz = slab_plane(a.g.z_off + gz, a.g, sz);
        }
        for (int i = tid; i < HY * HX; i += NT) {
            const int hy = i / HX, hx = i - hy * HX;
            const int gy = y0 - N + hy, gx = x0 - N + hx;
            int sy = 0, sx = 0;
            int s = sgz;
            if (RB) {   // no reflection: the basis does not vanish on the faces, ghosts are zero
                sy = gy;
                sx = gx;
                s = s && (unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx;
            } else {
                if (s) s *= reflect_index(gy, ny, sy);
                if (s) s *= reflect_index(gx, nx, sx);
            }
            T v = T(0);
            if (s) {
                const size_t o = ((size_t)sz * ny + sy) * nx + sx;
                if (!mask || mask[o]) {
                    T u;
                    if (MODE == MODE_CGP) {
                        const T r = a.in0[o];
                        const T zr = a.jvec  ? r * a.jvec[o]
                                     : a.jac ? r * jacobi_inv(a.jac, a.jn, sx, sy, sz)
                                             : r;
                        u = zr + beta * a.in1[o];
                    }
                    else if (MODE == MODE_MASS)
                        u = ld_io(a.in0, o, a.bf16io) + (a.in1 ? (T)a.s * ld_io(a.in1, o, a.bf16io) : T(0));
                    else if (MODE == MODE_OP) u = ld_io(a.in0, o, a.bf16io);
                    else u = a.in0[o];
                    v = s > 0 ? u : -u;
                }
            }
            dst[i] = v;
        }
    };

    for (int gz = zbase; gz < z0 + N; gz++) load_plane(gz);

    double acc0 = 0.0, acc1 = 0.0;
    for (int z = z0; z < z1; z++) {
        load_plane(z + N);
        __syncthreads();
        // z-sweep on the (TY + 2N) x (TX + 2N) halo tile
        const T* rzm = RB ? robin_row<T, N>(a.rb, 0, 2, z, nz) : nullptr;
        const T* rzk = RB ? robin_row<T, N>(a.rb, 1, 2, z, nz) : nullptr;
        for (int i = tid; i < HY * HX; i += NT) {
            T P = T(0), Q = T(0);
#pragma unroll
            for (int c = 0; c < L; c++) {
                const T v = ring[((z - N + c - zbase) % L) * (HY * HX) + i];
                P = fma(RB && rzm ? rzm[c] : a.c.M[2][c], v, P);
                if (!MASS_ONLY) Q = fma(RB && rzk ? rzk[c] : a.c.K[2][c], v, Q);
            }
            sP[i] = P;
            if (!MASS_ONLY) sQ[i] = Q;
        }
        __syncthreads();
        // y-sweep on the TY x (TX + 2N) tile
        for (int i = tid; i < TY * HX; i += NT) {
            const int ty = i / HX, hx = i - ty * HX;
            const T* rym = RB ? robin_row<T, N>(a.rb, 0, 1, y0 + ty, ny) : nullptr;
            const T* ryk = RB ? robin_row<T, N>(a.rb, 1, 1, y0 + ty, ny) : nullptr;
            T A = T(0), B = T(0);
#pragma unroll
            for (int b = 0; b < L; b++) {
                const T pv = sP[(ty + b) * HX + hx];
                const T my = RB && rym ? rym[b] : a.c.M[1][b];
                A = fma(my, pv, A);
                if (!MASS_ONLY) {
                    B = fma(RB && ryk ? ryk[b] : a.c.K[1][b], pv, B);
                    B = fma(my, sQ[(ty + b) * HX + hx], B);
                }
            }
            sA[i] = A;
            if (!MASS_ONLY) sS[i] = A + B;
        }
        __syncthreads();
        // x-sweep on the TY x TX output tile, fused epilogue
        for (int i = tid; i < TY * TX; i += NT) {
            const int ty = i / TX, tx = i - ty * TX;
            const int gy = y0 + ty, gx = x0 + tx;
            if (gx >= nx || gy >= ny) continue;
            const T* rxm = RB ? robin_row<T, N>(a.rb, 0, 0, gx, nx) : nullptr;
            const T* rxk = RB ? robin_row<T, N>(a.rb, 1, 0, gx, nx) : nullptr;
            T y = T(0);
#pragma unroll
            for (int c = 0; c < L; c++) {
                const T mx = RB && rxm ? rxm[c] : a.c.M[0][c];
                if (MASS_ONLY) {
                    y = fma(mx, sA[ty * HX + tx + c], y);
                } else {
                    y = fma(mx, sS[ty * HX + tx + c], y);
                    y = fma(RB && rxk ? rxk[c] : a.c.K[0][c], sA[ty * HX + tx + c], y);
                }
            }
            const size_t o = ((size_t)z * ny + gy) * nx + gx;
            const bool act = !mask || mask[o];
            if (!act) y = T(0);
            if (MODE == MODE_OP || MODE == MODE_MASS) {
                st_io(a.out0, o, y, a.bf16io);
            } else if (MODE == MODE_RES) {
                const T bv = act ? a.b[o] : T(0);
                const T r = bv - y;
                a.out0[o] = r;
                acc0 += (double)r * (double)r;
                acc1 += (double)bv * (double)bv;
            } else {  // MODE_CGP
                const T pn = ring[((z - zbase) % L) * (HY * HX) + (ty + N) * HX + (tx + N)];
                a.out1[o] = pn;
                a.out0[o] = y;
                a.xvec[o] = fma(alpha_prev, a.in1[o], a.xvec[o]);
                acc0 += (double)pn * (double)y;
            }
        }
        // The next plane's staging overwrites the ring slot of plane z - N, last read by the
        // z-sweep above (two barriers ago); sP/sQ and sA/sS are rewritten only after the next
        // barriers, so one barrier per phase suffices.
    }
    if (a.fin != FIN_NONE) grid_reduce2<NT>(acc0, acc1, a.partials, a.sc, a.fin, a.p_parity);
}

}  // namespace bsk
