// op_var.cuh -- the variable-coefficient operator y = A(d, m) x of arXiv:1904.03057, Eq. tensForm
// with the diffusion D(x) = sum d_m beta_m and the absorption mu_a(x) = sum m_m beta_m expanded
// in B-splines (section 2.3), computed on the fly (strategy (c) of section 2.4):
//
//   y_l = integral of dt D grad beta_l . grad u + mu_a beta_l u,
//
// with u the masked, odd-reflected solution expansion and D, mu_a even across the box faces.
// This is the triple sum sum_k sum_m x_k (dt d_m w^{klm} + m_m f^{klm}) of the paper, evaluated
// per knot interval ("cell") instead of per (k, m) pair: inside a cell every factor is one
// polynomial of degree n per axis, so a Gauss rule of Q = (3n + 2) / 2 points per axis
// integrates the degree-3n integrand exactly and the two forms agree up to rounding. With sum
// factorisation (one 1-D pass per axis) the cell form costs O(Q^3 (n + 1)) per node where the
// pair form costs O((2n + 1)^3 (n + 1)^3).
//
// One block owns a TT x TT (x, y) output tile and marches along z over the cells that touch its
// output planes [z0, z1). Per z-cell, with the N + 1 node planes of the cell in a ring:
//   A   z-pass: Q quad planes of cB = Bz c, cD = Dz c, dB = Bz d, mB = Bz m on the halo tile;
//   BC  one thread per (qz, y quad point) row: y-pass to five x-node values (U, dU/dy, dU/dz,
//       D, mu), x-pass to the Q points of each x cell, point fluxes dt D grad u and mu u times
//       the quadrature weight, and the transposed x-pass into the TT output columns (Xa, Xb,
//       Xc), all on rolling register windows;
//   D   one thread per (output column, quad plane): transposed y-pass;
//   E   one thread per output column: transposed z-pass into N + 1 plane accumulators; the
//       oldest plane is complete after its last cell and is written.
// The epilogue fuses the same CG vector work as the constant-coefficient kernels (residual,
// search-direction update, deferred x update, reductions).
#pragma once

#include "bsk_device.cuh"

namespace bsk {

constexpr int kVarMaxQ = 8;   // (3 * 5 + 2) / 2

// Gauss-point tables of one cell, shared by the three axes up to the derivative scale.
template <typename T>
struct VarTabs {
    T B[kVarMaxQ][kMaxDeg + 1];       // beta^n at Gauss point q for local basis t of the cell
    T D[3][kVarMaxQ][kMaxDeg + 1];    // beta^n' / h_axis (physical derivative), axis 0 = x
    T w[kVarMaxQ];                    // Gauss weights on the unit cell
    T Bw[kVarMaxQ][kMaxDeg + 1];      // w[q] B[q][t]: the transposed x-pass carries the x weight
    T Dxw[kVarMaxQ][kMaxDeg + 1];     // w[q] D[0][q][t]
};

template <typename T>
struct VarArgs {
    Geom g;
    VarTabs<T> t;
    T vol;            // hx hy hz (cell volume: the Jacobian of the weights)
    T dt;             // weight of the diffusion term
    const T* d;       // D coefficients at the (nz+2)(ny+2)(nx+2) nodes, faces included
    const T* m;       // mu_a coefficients, same layout
    const T* in0;     // x (OP, RES), r (CGP)
    const T* in1;     // p_old (CGP)
    T* out0;          // y (OP), r (RES), q = A p (CGP)
    T* out1;          // p (CGP)
    T* xvec;          // x, updated in place (CGP)
    const T* b;       // right-hand side (RES)
    const T* jvec;    // CGP: 1 / diag A per node (Jacobi), null = no preconditioner
    Scalars* sc;
    double* partials;
    int fin;
    int p_parity;
};

template <int N>
constexpr int var_q() { return (3 * N + 2) / 2; }

// Output tile side per element size and degree: the largest that keeps the three shared
// buffers within the 227 KB a block may hold.
template <typename T, int N>
constexpr int var_tile()
{
    if (sizeof(T) == 4) return N <= 3 ? 16 : N == 4 ? 12 : 10;
    return N == 1 ? 16 : N == 2 ? 12 : N <= 4 ? 8 : 4;
}

template <typename T, int N>
struct VarCfg {
    static constexpr int Q = var_q<N>();
    static constexpr int TT = var_tile<T, N>();
    static constexpr int H = TT + 2 * N;          // halo nodes per axis
    static constexpr int C = TT + N;              // cells per axis
    static constexpr int QC = Q * C;              // quad points per axis
    static constexpr int R = Q * QC;              // rows of stage BC per z-cell
    // X buffers are stored column-major, [field][qz][lx][RP]: the BC threads (consecutive rows)
    // store contiguously, and with RP = 2 (mod 32) the D warps (16 columns x 2 rows Q apart)
    // read 32 distinct banks
    static constexpr int RP = (QC + 29) / 32 * 32 + 2;
    static constexpr int PASSES = (R + 511) / 512;
    static constexpr int NT0 = ((R + PASSES - 1) / PASSES + 31) / 32 * 32;
    static constexpr int NT = NT0 < 64 ? 64 : NT0;
    static constexpr int NPT = (TT * TT + NT - 1) / NT;   // output columns per thread
    // quadrature weights folded into the y-passed fields and the transposed x tables (4 instead
    // of 8 products per point); above degree 3 the extra live values spill, so it is left out
    static constexpr bool FOLD = N <= 3;
    static constexpr size_t smem =
        sizeof(T) * ((size_t)3 * (N + 1) * H * H + (size_t)4 * Q * H * H + (size_t)3 * Q * TT * RP);
    static_assert(smem <= 227 * 1024, "variable-coefficient tile exceeds shared memory");
    // blocks per SM the register allocation must allow: two where two FP32 blocks' shared memory
    // fits (the FP64 kernels are bound by the FP64 pipe; capping their registers only spills)
    static constexpr int MINB = sizeof(T) == 4 && 2 * (smem + 1024) <= 228 * 1024 ? 2 : 1;
    static_assert(2 * Q * TT * TT <= 4 * Q * H * H, "the y-transposed planes reuse the quad planes");
};

// Coefficient node after even reflection across the faces at nodes 0 and n + 1. Positions more
// than one reflection away are clamped: only outputs outside the grid read them.
__device__ __forceinline__ int coef_node(int e, int n)
{
    if (e < 0) e = -e;
    if (e > n + 1) e = 2 * (n + 1) - e;
    return min(max(e, 0), n + 1);
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(VarCfg<T, N>::NT, VarCfg<T, N>::MINB) k_op_var(const __grid_constant__ VarArgs<T> a)
{
    using Cfg = VarCfg<T, N>;
    constexpr int Q = Cfg::Q, NB = N + 1, TT = Cfg::TT, H = Cfg::H, C = Cfg::C, QC = Cfg::QC;
    constexpr int NT = Cfg::NT, R = Cfg::R, NPT = Cfg::NPT, RP = Cfg::RP;
    constexpr bool FOLD = Cfg::FOLD;
    constexpr int HH = H * H, XS = Q * TT * RP;   // plane size, stride between X fields
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);   // [N + 1][3][HH]: c, d, m per node plane
    T* sZ = ring + (N + 1) * 3 * HH;            // [Q][4][HH]: cB, cD, dB, mB
    T* sX = sZ + Q * 4 * HH;                    // [3][Q][TT][RP]: Xa, Xb, Xc

    const int tid = threadIdx.x;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const uint8_t* __restrict__ mask = a.g.mask;

    T beta = T(0), alpha_prev = T(0);
    if (MODE == MODE_CGP) {
        if (*(volatile int*)&a.sc->done) return;  // uniform over the grid
        beta = (T)a.sc->beta;
        alpha_prev = (T)a.sc->alpha_prev;
    }

    const int x0 = blockIdx.x * TT, y0 = blockIdx.y * TT;
    const int z0 = blockIdx.z * a.g.tz;
    const int z1 = min(z0 + a.g.tz, nz);
    const int pz0 = z0 - N;                      // first node plane read by the block
    const int cpx = nx + 2, cpy = ny + 2;
    auto slot = [&](int gz) { return ring + ((gz - pz0) % (N + 1)) * (3 * HH); };

    // One node plane of the halo tile (solution value, D, mu_a) into registers, and from there
    // into its ring slot. The next plane is fetched before the long stages of the current cell
    // and stored at the start of the next one, so its loads are in flight meanwhile.
    constexpr int PRE = (HH + NT - 1) / NT;
    auto fetch_plane = [&](int gz, T (&pv)[PRE][3]) {
        int sz = 0;
        const int sgz = reflect_index(gz, nz, sz);
        const size_t ez = (size_t)coef_node(gz + 1, nz) * cpy;
#pragma unroll
        for (int k = 0; k < PRE; k++) {
            const int i = tid + k * NT;
            if (i >= HH) break;
            const int hy = i / H, hx = i - hy * H;
            const int gy = y0 - N + hy, gx = x0 - N + hx;
            int sy = 0, sx = 0;
            int s = sgz;
            if (s) s *= reflect_index(gy, ny, sy);
            if (s) s *= reflect_index(gx, nx, sx);
            T v = T(0);
            if (s) {
                const size_t o = ((size_t)sz * ny + sy) * nx + sx;
                const T u = MODE == MODE_CGP ? (a.jvec ? a.in0[o] * a.jvec[o] : a.in0[o]) + beta * a.in1[o]
                                             : a.in0[o];
                v = (mask && !mask[o]) ? T(0) : (s > 0 ? u : -u);
            }
            const size_t e = (ez + coef_node(gy + 1, ny)) * cpx + coef_node(gx + 1, nx);
            pv[k][0] = v;
            pv[k][1] = a.d[e];
            pv[k][2] = a.m[e];
        }
    };
    auto store_plane = [&](int gz, const T (&pv)[PRE][3]) {
        T* dst = slot(gz);
#pragma unroll
        for (int k = 0; k < PRE; k++) {
            const int i = tid + k * NT;
            if (i >= HH) break;
            dst[i] = pv[k][0];
            dst[HH + i] = pv[k][1];
            dst[2 * HH + i] = pv[k][2];
        }
    };

    // prefetching pays for FP32 from degree 3 up (1 %); for FP64 the values held across the
    // stages spill
    constexpr bool PREFETCH = N >= 3 && sizeof(T) == 4;
    T pre[PRE][3];
    for (int gz = pz0; gz < pz0 + N; gz++) {
        fetch_plane(gz, pre);
        store_plane(gz, pre);
    }
    if (PREFETCH) fetch_plane(pz0 + N, pre);

    T acc[NPT][NB];
#pragma unroll
    for (int k = 0; k < NPT; k++)
#pragma unroll
        for (int t = 0; t < NB; t++) acc[k][t] = T(0);
    double s0 = 0.0, s1 = 0.0;

    const int ncells = z1 - z0 + N;
    for (int kc = 0; kc < ncells; kc++) {
        const int pz = pz0 + kc;   // plane of local basis 0 of this z-cell
        __syncthreads();           // the previous epilogue read the slot reloaded here
        if (!PREFETCH) fetch_plane(pz + N, pre);
        store_plane(pz + N, pre);
        __syncthreads();
        if (PREFETCH && kc + 1 < ncells) fetch_plane(pz + N + 1, pre);
        // ---- A: z-pass on the halo tile ----
        for (int i = tid; i < Q * HH; i += NT) {
            const int qz = i / HH, k = i - qz * HH;
            T cB = T(0), cD = T(0), dB = T(0), mB = T(0);
#pragma unroll
            for (int t = 0; t < NB; t++) {
                const T* pl = slot(pz + t);
                const T bz = a.t.B[qz][t], dz = a.t.D[2][qz][t];
                const T c = pl[k];
                cB = fma(bz, c, cB);
                cD = fma(dz, c, cD);
                dB = fma(bz, pl[HH + k], dB);
                mB = fma(bz, pl[2 * HH + k], mB);
            }
            T* zq = sZ + qz * (4 * HH);
            zq[k] = cB;
            zq[HH + k] = cD;
            zq[2 * HH + k] = dB;
            zq[3 * HH + k] = mB;
        }
        __syncthreads();
        // ---- BC: per (qz, y quad point) row: y-pass, x-pass, fluxes, transposed x-pass ----
        for (int r = tid; r < R; r += NT) {
            const int qz = r / QC, yq = r - qz * QC;
            const int cy = yq / Q, qy = yq - cy * Q;
            const T* zq = sZ + qz * (4 * HH) + cy * H;
            T by[NB], dy[NB];
#pragma unroll
            for (int t = 0; t < NB; t++) {
                by[t] = a.t.B[qy][t];
                dy[t] = a.t.D[1][qy][t];
            }
            const T wyz = a.vol * a.t.w[qy] * a.t.w[qz];
            const T wyzdt = a.dt * wyz;
            // y-pass of node column hx: U, dU/dy, dU/dz (before the x-pass), D, mu
            auto ynode = [&](int hx, T (&v)[5]) {
#pragma unroll
                for (int f = 0; f < 5; f++) v[f] = T(0);
#pragma unroll
                for (int t = 0; t < NB; t++) {
                    const int k = t * H + hx;
                    const T cb = zq[k];
                    v[0] = fma(by[t], cb, v[0]);
                    v[1] = fma(dy[t], cb, v[1]);
                    v[2] = fma(by[t], zq[HH + k], v[2]);
                    v[3] = fma(by[t], zq[2 * HH + k], v[3]);
                    v[4] = fma(by[t], zq[3 * HH + k], v[4]);
                }
                if (FOLD) {   // the y and z weights (and dt) of the row's points, once per node
                    v[3] *= wyzdt;
                    v[4] *= wyz;
                }
            };
            T win[5][NB];   // y-passed node values of the current x cell: nodes cx .. cx + N
            T xo[3][NB];    // transposed x-pass accumulators of outputs cx - N .. cx
#pragma unroll
            for (int t = 0; t < N; t++) {
                T v[5];
                ynode(t, v);
#pragma unroll
                for (int f = 0; f < 5; f++) win[f][t] = v[f];
            }
#pragma unroll
            for (int f = 0; f < 3; f++)
#pragma unroll
                for (int t = 0; t < NB; t++) xo[f][t] = T(0);
            T* xrow = sX + (size_t)qz * TT * RP + yq;   // column lx at xrow[lx * RP]
            // unrolled by a multiple of the window length, the window shifts below are register
            // renames; up to degree 3 the whole cell loop is unrolled (measured 0.5-4 % faster;
            // above, the longer code measured 8-30 % slower)
            constexpr int UNROLL = N <= 3 ? C : NB;
#pragma unroll UNROLL
            for (int cx = 0; cx < C; cx++) {
                {
                    T v[5];
                    ynode(cx + N, v);
#pragma unroll
                    for (int f = 0; f < 5; f++) win[f][N] = v[f];
                }
#pragma unroll
                for (int qx = 0; qx < Q; qx++) {
                    T U = T(0), Ux = T(0), Uy = T(0), Uz = T(0), Dv = T(0), Mv = T(0);
#pragma unroll
                    for (int t = 0; t < NB; t++) {
                        const T bx = a.t.B[qx][t], dx = a.t.D[0][qx][t];
                        U = fma(bx, win[0][t], U);
                        Ux = fma(dx, win[0][t], Ux);
                        Uy = fma(bx, win[1][t], Uy);
                        Uz = fma(bx, win[2][t], Uz);
                        Dv = fma(bx, win[3][t], Dv);
                        Mv = fma(bx, win[4][t], Mv);
                    }
                    // point fluxes dt D grad u and mu u times the point weight; with FOLD the y, z
                    // weights are already in Dv, Mv and the x weight is in the Bw, Dxw tables
                    T G = Dv, S = Mv * U;
                    if (!FOLD) {
                        const T wq = a.t.w[qx];
                        G = (wq * wyzdt) * Dv;
                        S = (wq * wyz) * S;
                    }
                    const T Fx = G * Ux, Fy = G * Uy, Fz = G * Uz;
#pragma unroll
                    for (int t = 0; t < NB; t++) {
                        const T bw = FOLD ? a.t.Bw[qx][t] : a.t.B[qx][t];
                        const T dw = FOLD ? a.t.Dxw[qx][t] : a.t.D[0][qx][t];
                        xo[0][t] = fma(dw, Fx, fma(bw, S, xo[0][t]));
                        xo[1][t] = fma(bw, Fy, xo[1][t]);
                        xo[2][t] = fma(bw, Fz, xo[2][t]);
                    }
                }
                // output cx - N has now received all its cells
                const int lx = cx - N;
                if (lx >= 0 && lx < TT) {
                    xrow[lx * RP] = xo[0][0];
                    xrow[XS + lx * RP] = xo[1][0];
                    xrow[2 * XS + lx * RP] = xo[2][0];
                }
#pragma unroll
                for (int f = 0; f < 3; f++) {
#pragma unroll
                    for (int t = 0; t < N; t++) xo[f][t] = xo[f][t + 1];
                    xo[f][N] = T(0);
                }
#pragma unroll
                for (int f = 0; f < 5; f++)
#pragma unroll
                    for (int t = 0; t < N; t++) win[f][t] = win[f][t + 1];
            }
        }
        __syncthreads();
        // ---- D: transposed y-pass per (output column, quad plane), all threads; the results go
        // to sY, which reuses sZ (read for the last time in BC) ----
        T* sY = sZ;   // [2][Q][TT * TT]: Ya, Yc
        for (int i = tid; i < Q * TT * TT; i += NT) {
            const int qz = i / (TT * TT), node = i - qz * (TT * TT);
            const int ly = node / TT, lx = node - ly * TT;
            T Ya = T(0), Yc = T(0);
#pragma unroll
            for (int t = 0; t < NB; t++) {
                const T* xa = sX + ((size_t)qz * TT + lx) * RP + (ly + N - t) * Q;
#pragma unroll
                for (int qy = 0; qy < Q; qy++) {
                    const T b = a.t.B[qy][t], d = a.t.D[1][qy][t];
                    Ya = fma(b, xa[qy], fma(d, xa[XS + qy], Ya));
                    Yc = fma(b, xa[2 * XS + qy], Yc);
                }
            }
            sY[i] = Ya;
            sY[Q * TT * TT + i] = Yc;
        }
        __syncthreads();
        // ---- E: transposed z-pass into the plane accumulators of each output column ----
#pragma unroll
        for (int k = 0; k < NPT; k++) {
            const int node = tid + k * NT;
            if (node < TT * TT) {
#pragma unroll
                for (int qz = 0; qz < Q; qz++) {
                    const T Ya = sY[qz * TT * TT + node], Yc = sY[(Q + qz) * TT * TT + node];
#pragma unroll
                    for (int t = 0; t < NB; t++)
                        acc[k][t] = fma(a.t.B[qz][t], Ya, fma(a.t.D[2][qz][t], Yc, acc[k][t]));
                }
            }
        }
        // ---- epilogue: plane pz has received all its cells ----
        if (pz >= z0 && pz < z1) {
#pragma unroll
            for (int k = 0; k < NPT; k++) {
                const int node = tid + k * NT;
                const int ly = node / TT, lx = node - ly * TT;
                const int gy = y0 + ly, gx = x0 + lx;
                if (node < TT * TT && gx < nx && gy < ny) {
                    const size_t o = ((size_t)pz * ny + gy) * nx + gx;
                    const bool act = !mask || mask[o];
                    const T y = act ? acc[k][0] : T(0);
                    if (MODE == MODE_OP) {
                        a.out0[o] = y;
                    } else if (MODE == MODE_RES) {
                        const T bv = act ? a.b[o] : T(0);
                        const T r = bv - y;
                        a.out0[o] = r;
                        s0 += (double)r * (double)r;
                        s1 += (double)bv * (double)bv;
                    } else {  // MODE_CGP
                        const T pn = slot(pz)[(ly + N) * H + (lx + N)];
                        a.out1[o] = pn;
                        a.out0[o] = y;
                        a.xvec[o] = fma(alpha_prev, a.in1[o], a.xvec[o]);
                        s0 += (double)pn * (double)y;
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NPT; k++) {
#pragma unroll
            for (int t = 0; t < N; t++) acc[k][t] = acc[k][t + 1];
            acc[k][N] = T(0);
        }
    }
    if (a.fin != FIN_NONE) grid_reduce2<NT>(s0, s1, a.partials, a.sc, a.fin, a.p_parity);
}

}  // namespace bsk
