// bsk_device.cuh -- device-side types and helpers shared by the operator and vector kernels.
//
// The operator is the constant-coefficient case of Eq. tensForm (arXiv:1904.03057, section 2.4):
// y = Mz My Mx x + dt (Kz My Mx + Mz Ky Mx + Mz My Kx) x over odd-reflected, masked coefficients.
// The CG recurrences follow the conjugate gradient stage of section 2.5.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bsk {

constexpr int kMaxDeg = 5;
constexpr int kMaxTaps = 2 * kMaxDeg + 1;

// Output tile of the general operator kernel (x, y) and its block size.
constexpr int kGenTX = 32, kGenTY = 16, kGenNT = 256;

// Finalisation performed by the last block of a reducing kernel.
enum Fin : int {
    FIN_NONE = 0,
    FIN_RES_INIT = 1,   // CG start: rr = s0, bb = s1, decide trivial convergence
    FIN_RES_TRUE = 2,   // true residual after a solve: rr_true = s0, bb_true = s1
    FIN_CGP = 3,        // pq = s0 -> alpha
    FIN_UPD = 4,        // rr_new = s0 -> beta, convergence, iteration count
    FIN_NORM = 5,       // rr_true = s0
    FIN_CG1 = 6,        // single-pass CG: s0 = r.r, s1 = p.Ap, s2 = Ap.Ap -> alpha, beta, status
    FIN_PC_INIT = 7,    // preconditioned CG start: rz = s0 (r.z, z = r / diag A)
    FIN_UPD_PC = 8,     // preconditioned update: rr_new = s0 (convergence), rz_new = s1 -> beta
};

// Operator kernel modes.
enum OpMode : int {
    MODE_OP = 0,    // y = A x
    MODE_MASS = 1,  // y = M (x + s * x2)    (right-hand side of an implicit Euler step)
    MODE_RES = 2,   // r = b - A x, reductions r.r and b.b
    MODE_CGP = 3,   // p = r + beta p_old; x += alpha_prev p_old; q = A p; reduction p.q
};

// Modes of the TMA operator kernel (op_tma.cuh): y = A x; r = b - A x; one whole CG iteration.
enum TmaMode : int { TMODE_OP = 0, TMODE_RES = 1, TMODE_CG = 2 };

// CG state kept on the device; all scalars in FP64.
struct Scalars {
    double rr;          // r.r of the current residual
    double bb;          // b.b
    double pq;          // p.Ap of the current iteration
    double alpha;       // step length of the current iteration
    double alpha_prev;  // step length whose x update is still pending
    double beta;        // coefficient of the next search direction
    double tol2;        // tol^2 (relative to b.b)
    double best_rr;     // smallest rr seen (stall detection)
    double rr_true;     // reductions of the last true-residual / norm pass
    double bb_true;
    int iter;           // completed iterations
    int max_iter;
    int done;           // non-zero once the iteration has stopped
    int status;         // 0 converged, 1 max_iter, 2 stalled, -5 breakdown
    int since_best;
    int stall_window;
    int p_cur;          // which ping-pong buffer holds the latest search direction
    int zero_b;         // b == 0: the solution is x = 0
    unsigned int counter;  // arrival counter of the last-block reduction
    int pass;           // single-pass CG: passes completed (pass m produces x_m, r_m)
    double rz;          // preconditioned CG: r.z of the current residual (z = r / diag A)
    int pc;             // non-zero: Jacobi-preconditioned CG (alpha and beta from rz)
    double beta_prev;   // single-pass CG: the coefficient before `beta` (rebuilds r from two p)
};

// Per-axis kernels in compute precision: M[d][j + n], K[d][j + n] with K already scaled by dt.
// Axis 0 = x, 1 = y, 2 = z.
template <typename C>
struct Coef {
    C M[3][kMaxTaps];
    C K[3][kMaxTaps];
};

struct Geom {
    int nx, ny, nz;
    int tz;                 // output planes per block along z
    const uint8_t* mask;    // node mask (nullptr = whole box)
    // z-slab of a larger grid (MODE_OP only): the nz local planes are global planes
    // z_off .. z_off + nz - 1 of nz_glob, and the input carries zpad extra planes on each side
    // (input plane i is global plane z_off - zpad + i). Odd reflection applies at the global
    // faces only. A whole grid has z_off = 0, nz_glob = nz, zpad = 0.
    int z_off, nz_glob, zpad;
};


// Index of array position a (0-based) after odd reflection about the faces at -1 and N.
// Returns +1 (interior, src = a), -1 (ghost, src = mirror image), 0 (face or beyond: zero).
__device__ __forceinline__ int reflect_index(int a, int N, int& src)
{
    if ((unsigned)a < (unsigned)N) { src = a; return 1; }
    int r = a < 0 ? -2 - a : 2 * N - a;
    if ((unsigned)r >= (unsigned)N) return 0;
    src = r;
    return -1;
}

// Input plane (counted in the input array) that holds global plane g of a z-slab after odd
// reflection about the global faces; returns the sign (+1, -1, 0 = face or beyond).
__device__ __forceinline__ int slab_plane(int g, const Geom& geo, int& src)
{
    int sg = 0;
    const int s = reflect_index(g, geo.nz_glob, sg);
    src = sg - geo.z_off + geo.zpad;
    return s;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of two values; the result is valid in thread 0. sred needs 2 * warps doubles.
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sred)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { sred[warp] = a; sred[NW + warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int w = 0; w < NW; w++) { sa += sred[w]; sb += sred[NW + w]; }
        a = sa;
        b = sb;
    }
}

__device__ __forceinline__ void finalize(Scalars* sc, int fin, double s0, double s1, int p_parity)
{
    switch (fin) {
    case FIN_RES_INIT:
        sc->rr = s0;
        sc->bb = s1;
        sc->best_rr = s0;
        sc->since_best = 0;
        sc->iter = 0;
        sc->alpha = 0.0;
        sc->alpha_prev = 0.0;
        sc->beta = 0.0;
        sc->beta_prev = 0.0;
        sc->p_cur = 0;
        sc->zero_b = 0;
        sc->done = 0;
        sc->status = 0;
        if (!isfinite(s0) || !isfinite(s1)) { sc->done = 1; sc->status = -5; }
        else if (s1 == 0.0) { sc->done = 1; sc->zero_b = 1; }
        else if (s0 <= sc->tol2 * s1) { sc->done = 1; }
        break;
    case FIN_RES_TRUE:
        sc->rr_true = s0;
        sc->bb_true = s1;
        break;
    case FIN_NORM:
        sc->rr_true = s0;
        break;
    case FIN_CGP:
        sc->pq = s0;
        sc->p_cur = p_parity;
        if (!(s0 > 0.0) || !isfinite(s0)) {
            sc->done = 1;
            sc->status = -5;
            sc->alpha = 0.0;
            sc->alpha_prev = 0.0;
        } else {
            sc->alpha = (sc->pc ? sc->rz : sc->rr) / s0;
            sc->alpha_prev = sc->alpha;
        }
        break;
    case FIN_PC_INIT:
        sc->rz = s0;
        if (!isfinite(s0)) { sc->done = 1; sc->status = -5; }
        break;
    case FIN_UPD:
    case FIN_UPD_PC: {
        const double rr_new = s0;
        sc->iter += 1;
        if (!isfinite(rr_new) || (fin == FIN_UPD_PC && !isfinite(s1))) { sc->done = 1; sc->status = -5; break; }
        if (rr_new <= sc->tol2 * sc->bb) { sc->done = 1; sc->status = 0; }
        else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = 1; }
        else if (rr_new < sc->best_rr) { sc->best_rr = rr_new; sc->since_best = 0; }
        else if (sc->stall_window > 0 && ++sc->since_best >= sc->stall_window) {
            sc->done = 1;
            sc->status = 2;
        }
        if (fin == FIN_UPD_PC) {
            sc->beta = s1 / sc->rz;
            sc->rz = s1;
        } else {
            sc->beta = rr_new / sc->rr;
        }
        sc->rr = rr_new;
        break;
    }
    default:
        break;
    }
}

// Single-pass CG finaliser (one grid reduction per iteration). Pass m has produced r_m, x_m,
// p_m and q_m = A p_m with s0 = r_m.r_m, s1 = p_m.q_m, s2 = q_m.q_m. The next step length is
// alpha_m = rr_m / pq_m, and ||r_{m+1}||^2 = ||r_m - alpha_m q_m||^2 is predicted as
// alpha_m^2 qq_m - rr_m (using r_m.q_m = p_m.q_m, exact in exact arithmetic), which gives
// beta_m without a second reduction; rr itself is always the exactly reduced value.
__device__ __forceinline__ void finalize_cg1(Scalars* sc, double rr, double pq, double qq)
{
    const int m = sc->pass;
    sc->pass = m + 1;
    sc->iter = m;
    sc->rr = rr;
    sc->pq = pq;
    if (!isfinite(rr) || !isfinite(pq) || !isfinite(qq)) { sc->done = 1; sc->status = -5; return; }
    if (rr <= sc->tol2 * sc->bb) { sc->done = 1; sc->status = 0; return; }
    if (m >= sc->max_iter) { sc->done = 1; sc->status = 1; return; }
    if (!(pq > 0.0)) { sc->done = 1; sc->status = -5; return; }
    if (rr < sc->best_rr) { sc->best_rr = rr; sc->since_best = 0; }
    else if (sc->stall_window > 0 && ++sc->since_best >= sc->stall_window) {
        sc->done = 1;
        sc->status = 2;
        return;
    }
    const double alpha = rr / pq;
    double rr_next = alpha * alpha * qq - rr;
    if (rr_next < 0.0) rr_next = 0.0;
    sc->alpha = alpha;
    sc->beta_prev = sc->beta;
    sc->beta = rr_next / rr;
}

// Deterministic grid reduction of K values: each block stores its partial sums, the last block
// to arrive adds all partials in block order and runs the finaliser. partials holds K * nblocks
// doubles. Must be called by every thread of the block (contains __syncthreads).
template <int NT, int K>
__device__ void grid_reduce_k(double (&v)[K], double* partials, Scalars* sc, int fin)
{
    constexpr int NW = NT / 32;
    __shared__ double sred[K * NW];
    __shared__ int s_last;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = warp_sum(v[k]);
        if (lane == 0) sred[k * NW + warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int w = 0; w < NW; w++) s += sred[k * NW + w];
            partials[k * nblocks + bid] = s;
        }
        __threadfence();
        unsigned prev = atomicAdd(&sc->counter, 1u);
        s_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    for (unsigned i = threadIdx.x; i < nblocks; i += NT)
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] += __ldcg(partials + k * nblocks + i);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = warp_sum(acc[k]);
        if (lane == 0) sred[k * NW + warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[K];
        for (int k = 0; k < K; k++) {
            tot[k] = 0.0;
            for (int w = 0; w < NW; w++) tot[k] += sred[k * NW + w];
        }
        if (fin == FIN_CG1) finalize_cg1(sc, tot[0], K > 1 ? tot[1] : 0.0, K > 2 ? tot[2] : 0.0);
        else finalize(sc, fin, tot[0], K > 1 ? tot[1] : 0.0, 0);
        sc->counter = 0;
        __threadfence();
    }
}

// Deterministic two-value grid reduction: each block stores its partial sums, the last block to
// arrive adds all partials in block order and runs the finaliser. partials holds 2 * nblocks
// doubles. Must be called by every thread of the block (contains __syncthreads).
template <int NT>
__device__ void grid_reduce2(double a, double b, double* partials, Scalars* sc, int fin,
                             int p_parity)
{
    __shared__ double sred[2 * (NT / 32)];
    __shared__ int s_last;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_sum2<NT>(a, b, sred);
    if (threadIdx.x == 0) {
        partials[bid] = a;
        partials[nblocks + bid] = b;
        __threadfence();
        unsigned prev = atomicAdd(&sc->counter, 1u);
        s_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (unsigned i = threadIdx.x; i < nblocks; i += NT) {
        sa += __ldcg(partials + i);
        sb += __ldcg(partials + nblocks + i);
    }
    __syncthreads();  // sred reuse
    block_sum2<NT>(sa, sb, sred);
    if (threadIdx.x == 0) {
        finalize(sc, fin, sa, sb, p_parity);
        sc->counter = 0;
        __threadfence();
    }
}

}  // namespace bsk
