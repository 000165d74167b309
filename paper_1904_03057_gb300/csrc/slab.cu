// slab.cu -- CG vector passes of a z-slab of a grid split across devices (section 3 of
// arXiv:1904.03057 distributes the unknowns over GPUs; here the split is along z).
//
// Each device holds nz local planes of the global grid plus n halo planes of the search
// direction on each side. One CG iteration (section 2.5) on a slab is
//   exchange the halo planes of p with the neighbouring slabs
//   q = A p over the local planes                 (general operator kernel, z-slab geometry)
//   local p.q                                     slab_dot          -> all-reduce
//   alpha = rr / pq; x += alpha p; r -= alpha q;  slab_update       -> all-reduce of r.r
//   beta = rr_new / rr; p = r + beta p            slab_direction    (convergence test)
// The scalars live in a small device array (layout BSK_SLAB_* of bsk.h) so that the all-reduces
// (NCCL on device buffers, or any host routine) act on it in place between the passes. Every
// pass returns at once when the solve has finished, so iterations queued past convergence leave
// x and r unchanged. Reductions are deterministic: per-block partial sums, added in block order
// by the last block to finish, which also runs the scalar bookkeeping of the pass.
#include "bsk_launch.h"
#include "vec_kernels.cuh"
#include "bsk.h"

namespace bsk {

namespace {

constexpr int kSlabNT = 256;
constexpr int kSlabMaxGrid = 2048;   // partial-sum buffers hold 2 * kSlabMaxGrid doubles

enum SlabPhase { SP_BEGIN, SP_DOT, SP_UPDATE, SP_FIRST, SP_DIRECTION };

int slab_grid(size_t len)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    const size_t want = (len + kSlabNT - 1) / kSlabNT;
    size_t g = want < (size_t)sms * 8 ? want : (size_t)sms * 8;
    if (g > (size_t)kSlabMaxGrid) g = kSlabMaxGrid;
    return g < 1 ? 1 : (int)g;
}

__device__ __forceinline__ bool slab_done(const double* s) { return *(volatile const double*)&s[BSK_SLAB_DONE] != 0.0; }

__device__ void slab_finish(double* s, int phase, double v0, double v1)
{
    switch (phase) {
    case SP_BEGIN:   // local r.r and b.b of the starting residual
        s[BSK_SLAB_RR_NEW] = v0;
        s[BSK_SLAB_BB] = v1;
        break;
    case SP_DOT:     // local p.q
        s[BSK_SLAB_PQ] = v0;
        break;
    case SP_UPDATE: {
        const double pq = s[BSK_SLAB_PQ];
        if (!(pq > 0.0) || !isfinite(pq)) {   // A p vanished or overflowed: breakdown
            s[BSK_SLAB_DONE] = 1.0;
            s[BSK_SLAB_STATUS] = -5.0;
        }
        s[BSK_SLAB_RR_NEW] = v0;              // local r.r of the updated residual
        break;
    }
    case SP_FIRST:
    case SP_DIRECTION: {
        const double rr = s[BSK_SLAB_RR_NEW], bb = s[BSK_SLAB_BB];
        double it = s[BSK_SLAB_ITER];
        if (phase == SP_DIRECTION) s[BSK_SLAB_ITER] = it = it + 1.0;
        s[BSK_SLAB_RR] = rr;
        if (!isfinite(rr) || !isfinite(bb)) { s[BSK_SLAB_DONE] = 1.0; s[BSK_SLAB_STATUS] = -5.0; }
        else if (rr <= s[BSK_SLAB_TOL2] * bb) { s[BSK_SLAB_DONE] = 1.0; s[BSK_SLAB_STATUS] = 0.0; }
        else if (it >= s[BSK_SLAB_MAX_ITER]) { s[BSK_SLAB_DONE] = 1.0; s[BSK_SLAB_STATUS] = 1.0; }
        break;
    }
    default:
        break;
    }
}

// Adds the per-thread values of the grid in block order and runs the phase's bookkeeping in the
// last block to arrive. Called by every thread of every block.
__device__ void slab_reduce(double v0, double v1, double* partials, unsigned* ctr, double* s, int phase)
{
    __shared__ double sred[2 * (kSlabNT / 32)];
    __shared__ int s_last;
    const unsigned nb = gridDim.x;
    block_sum2<kSlabNT>(v0, v1, sred);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v0;
        partials[nb + blockIdx.x] = v1;
        __threadfence();
        s_last = atomicAdd(ctr, 1u) == nb - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned i = threadIdx.x; i < nb; i += kSlabNT) {
        a += __ldcg(partials + i);
        b += __ldcg(partials + nb + i);
    }
    __syncthreads();
    block_sum2<kSlabNT>(a, b, sred);
    if (threadIdx.x == 0) {
        slab_finish(s, phase, a, b);
        *ctr = 0u;
        __threadfence();
    }
}

// r = b - A x (A x given), p = r on the local planes; local r.r and b.b.
template <typename T>
__global__ void __launch_bounds__(kSlabNT) k_slab_begin(const T* __restrict__ b, const T* __restrict__ ax,
                                                        T* __restrict__ r, T* __restrict__ p, size_t len,
                                                        double* s, double* partials, unsigned* ctr)
{
    SqSum<T> rr, bb;
    for (size_t i = blockIdx.x * (size_t)kSlabNT + threadIdx.x; i < len; i += (size_t)gridDim.x * kSlabNT) {
        const T bv = b[i];
        const T v = bv - ax[i];
        r[i] = v;
        p[i] = v;
        rr.add(v);
        bb.add(bv);
    }
    slab_reduce(rr.value(), bb.value(), partials, ctr, s, SP_BEGIN);
}

// Local p.q.
template <typename T>
__global__ void __launch_bounds__(kSlabNT) k_slab_dot(const T* __restrict__ p, const T* __restrict__ q, size_t len,
                                                      double* s, double* partials, unsigned* ctr)
{
    if (slab_done(s)) return;
    TermSum<T> pq;
    for (size_t i = blockIdx.x * (size_t)kSlabNT + threadIdx.x; i < len; i += (size_t)gridDim.x * kSlabNT)
        pq.add(p[i] * q[i]);
    slab_reduce(pq.value(), 0.0, partials, ctr, s, SP_DOT);
}

// alpha = rr / pq (both all-reduced); x += alpha p, r -= alpha q; local r.r of the new r.
template <typename T>
__global__ void __launch_bounds__(kSlabNT) k_slab_update(T* __restrict__ x, T* __restrict__ r,
                                                         const T* __restrict__ p, const T* __restrict__ q,
                                                         size_t len, double* s, double* partials, unsigned* ctr)
{
    if (slab_done(s)) return;
    const double pq = s[BSK_SLAB_PQ];
    const bool ok = pq > 0.0 && isfinite(pq);
    const T alpha = ok ? (T)(s[BSK_SLAB_RR] / pq) : T(0);
    SqSum<T> rr;
    if (ok)
        for (size_t i = blockIdx.x * (size_t)kSlabNT + threadIdx.x; i < len; i += (size_t)gridDim.x * kSlabNT) {
            x[i] = fma(alpha, p[i], x[i]);
            const T v = fma(-alpha, q[i], r[i]);
            r[i] = v;
            rr.add(v);
        }
    slab_reduce(rr.value(), 0.0, partials, ctr, s, SP_UPDATE);
}

// p = r + beta p with beta = rr_new / rr (all-reduced), or p = r on the first pass; then the
// convergence test on rr_new.
template <typename T>
__global__ void __launch_bounds__(kSlabNT) k_slab_direction(const T* __restrict__ r, T* __restrict__ p, size_t len,
                                                            int first, double* s, double* partials, unsigned* ctr)
{
    if (slab_done(s)) return;
    const T beta = first ? T(0) : (T)(s[BSK_SLAB_RR_NEW] / s[BSK_SLAB_RR]);
    for (size_t i = blockIdx.x * (size_t)kSlabNT + threadIdx.x; i < len; i += (size_t)gridDim.x * kSlabNT)
        p[i] = fma(beta, p[i], r[i]);
    slab_reduce(0.0, 0.0, partials, ctr, s, first ? SP_FIRST : SP_DIRECTION);
}

}  // namespace

template <typename T>
cudaError_t slab_pass(int pass, const SlabVectors& v, size_t len, double* s, double* partials, unsigned* ctr,
                      cudaStream_t st)
{
    const int g = slab_grid(len);
    const T* b = static_cast<const T*>(v.b);
    const T* ax = static_cast<const T*>(v.ax);
    const T* q = static_cast<const T*>(v.q);
    T* x = static_cast<T*>(v.x);
    T* r = static_cast<T*>(v.r);
    T* p = static_cast<T*>(v.p);
    switch (pass) {
    case SLAB_BEGIN: k_slab_begin<T><<<g, kSlabNT, 0, st>>>(b, ax, r, p, len, s, partials, ctr); break;
    case SLAB_DOT: k_slab_dot<T><<<g, kSlabNT, 0, st>>>(p, q, len, s, partials, ctr); break;
    case SLAB_UPDATE: k_slab_update<T><<<g, kSlabNT, 0, st>>>(x, r, p, q, len, s, partials, ctr); break;
    case SLAB_FIRST: k_slab_direction<T><<<g, kSlabNT, 0, st>>>(r, p, len, 1, s, partials, ctr); break;
    case SLAB_DIRECTION: k_slab_direction<T><<<g, kSlabNT, 0, st>>>(r, p, len, 0, s, partials, ctr); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t slab_pass<float>(int, const SlabVectors&, size_t, double*, double*, unsigned*, cudaStream_t);
template cudaError_t slab_pass<double>(int, const SlabVectors&, size_t, double*, double*, unsigned*, cudaStream_t);

size_t slab_partials_doubles() { return 2 * (size_t)kSlabMaxGrid; }

}  // namespace bsk
