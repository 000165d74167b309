// fcg.cu -- flexible conjugate gradients with the learned preconditioner (fcg_solve).
//
// FCG(1) (truncated flexible CG, one previous direction kept conjugate), preconditioned by
//   z_k = ||r_k|| N(r_k / ||r_k||) / (hx hy hz)          (the network, net.cu)
//   beta_k = -(z_k . q_{k-1}) / (p_{k-1} . q_{k-1}),   p_k = z_k + beta_k p_{k-1}
//   q_k = A p_k,   alpha_k = (r_k . p_k) / (p_k . q_k),   x += alpha_k p_k,   r -= alpha_k q_k
// run as the inner FP32 solver of iterative refinement (the FP64 true residual b - A x outside
// is the arbiter of convergence). An iteration whose network direction is not a descent
// direction (z . r <= 0) takes z = r for that iteration only; a non-finite network output or a
// residual that stops improving makes the iteration fall back to plain CG (z = r) for the rest
// of the inner solve. All scalars stay on the device; the host
// polls the status every few iterations. The paper's solver stage is plain CG (section 2.5);
// the preconditioner is the workload's addition.
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>

#include "bsk.h"
#include "bsk_launch.h"

using bsk::Scalars;

namespace {

constexpr int NT = 256;

// Device state of the inner FCG iteration (one per handle).
struct FcgState {
    double rr, bb, tol2;
    double pq_prev;      // p_{k-1} . q_{k-1}
    double beta, alpha;
    double best_rr;
    double zscale;       // ||r_k||: the network sees r / ||r||
    double out_scale;    // the network's output unit: z = ||r|| out_scale N(r / ||r||) + jac r
    double jac;          // Jacobi part of the preconditioner: 1 / A_ii
    int unit_input;      // linear network: it sees r itself (z = out_scale N(r)), no normalisation
    int iter, max_iter, done, status;
    int use_r;           // 1: plain CG direction for the rest of the solve (fallback engaged)
    int dir_r;           // 1: this iteration's direction is r (use_r, or z . r <= 0 this time)
    int rejected;        // iterations whose network direction was replaced by r
    int fallback_iter;   // iteration at which the fallback engaged, -1 if never
    int since_best, stall_window;
    int first;           // no previous direction yet
    unsigned int counter;
    int pad;
};

// Per-thread compensated FP32 sum (Kahan): the element products stay on the FP32 pipes (GB300
// runs FP64 at 1/62 of the FP32 rate); each thread's sum is widened to FP64 once for the
// deterministic block and grid reduction.
struct FSum {
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

template <int K, typename F>
__device__ void reduce_then(double (&v)[K], double* partials, unsigned int* counter, F fin)
{
    __shared__ double sred[K * (NT / 32)];
    __shared__ int s_last;
    const unsigned nb = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sred[k * (NT / 32) + warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; w++) s += sred[k * (NT / 32) + w];
            partials[k * nb + blockIdx.x] = s;
        }
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == nb - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    for (unsigned i = threadIdx.x; i < nb; i += NT)
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] += __ldcg(partials + k * nb + i);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sred[k * (NT / 32) + warp] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[K];
        for (int k = 0; k < K; k++) {
            tot[k] = 0.0;
            for (int w = 0; w < NT / 32; w++) tot[k] += sred[k * (NT / 32) + w];
        }
        fin(tot);
        *counter = 0;
        __threadfence();
    }
}

#define GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < (n); i += (size_t)gridDim.x * NT)

// start from x = 0: r = mask(b), x = 0, rr = bb = r.r
__global__ void __launch_bounds__(NT) k_fcg_init(const float* __restrict__ b, float* __restrict__ r,
                                                 float* __restrict__ x, size_t n, const uint8_t* __restrict__ mask,
                                                 FcgState* st, double* partials)
{
    FSum acc;
    GRID_STRIDE(i, n)
    {
        const float v = (!mask || mask[i]) ? b[i] : 0.f;
        r[i] = v;
        x[i] = 0.f;
        acc.add(v * v);
    }
    double v1[1] = {acc.value()};
    reduce_then<1>(v1, partials, &st->counter, [&](double* t) {
        st->rr = t[0];
        st->bb = t[0];
        st->best_rr = t[0];
        st->iter = 0;
        st->first = 1;
        st->since_best = 0;
        st->done = (t[0] == 0.0 || t[0] <= st->tol2 * t[0]) ? 1 : 0;
        st->status = isfinite(t[0]) ? 0 : -5;
        if (!isfinite(t[0])) st->done = 1;
        st->zscale = sqrt(t[0]);
    });
}

// network input: rn = r / ||r||
__global__ void __launch_bounds__(NT) k_fcg_normalise(const float* __restrict__ r, float* __restrict__ rn, size_t n,
                                                      const FcgState* st)
{
    if (st->done) return;
    const float inv = st->zscale > 0 ? (float)(1.0 / st->zscale) : 0.f;
    GRID_STRIDE(i, n) rn[i] = r[i] * inv;
}

// z = ||r|| zn; reductions z.q_prev, z.r, r.q_prev -> beta and the choice of direction
__global__ void __launch_bounds__(NT) k_fcg_direction(const float* __restrict__ zn, float* __restrict__ z,
                                                      const float* __restrict__ r, const float* __restrict__ q,
                                                      size_t n, FcgState* st, double* partials)
{
    if (st->done) return;
    const float s = (float)((st->unit_input ? 1.0 : st->zscale) * st->out_scale);
    const float jac = (float)st->jac;
    FSum zq, zr, rq;
    GRID_STRIDE(i, n)
    {
        const float zv = fmaf(s, zn[i], jac * r[i]);   // jac = 0 unless a fixed diagonal part is set
        z[i] = zv;
        zq.add(zv * q[i]);
        zr.add(zv * r[i]);
        rq.add(r[i] * q[i]);
    }
    double v3[3] = {zq.value(), zr.value(), rq.value()};
    reduce_then<3>(v3, partials, &st->counter, [&](double* t) {
        const bool finite = isfinite(t[0]) && isfinite(t[1]);
        if (!finite && !st->use_r) {
            st->use_r = 1;
            st->fallback_iter = st->iter;
        }
        // a network direction with z . r <= 0 is no descent direction: use r this time
        st->dir_r = st->use_r || !(t[1] > 0.0);
        if (st->dir_r && !st->use_r) st->rejected += 1;
        if (st->first) st->beta = 0.0;
        else st->beta = -(st->dir_r ? t[2] : t[0]) / st->pq_prev;
    });
}

// p = d + beta p with d = r (plain CG) or z (network)
__global__ void __launch_bounds__(NT) k_fcg_p(const float* __restrict__ z, const float* __restrict__ r,
                                              float* __restrict__ p, size_t n, const FcgState* st)
{
    if (st->done) return;
    const float beta = (float)st->beta;
    const float* d = st->dir_r ? r : z;
    if (st->first) {
        GRID_STRIDE(i, n) p[i] = d[i];
    } else {
        GRID_STRIDE(i, n) p[i] = fmaf(beta, p[i], d[i]);
    }
}

// alpha = (r.p) / (p.q)
__global__ void __launch_bounds__(NT) k_fcg_alpha(const float* __restrict__ r, const float* __restrict__ p,
                                                  const float* __restrict__ q, size_t n, FcgState* st,
                                                  double* partials)
{
    if (st->done) return;
    FSum rp, pq;
    GRID_STRIDE(i, n)
    {
        rp.add(r[i] * p[i]);
        pq.add(p[i] * q[i]);
    }
    double v2[2] = {rp.value(), pq.value()};
    reduce_then<2>(v2, partials, &st->counter, [&](double* t) {
        if (!(t[1] > 0.0) || !isfinite(t[0]) || !isfinite(t[1])) {
            st->done = 1;
            st->status = -5;
            st->alpha = 0.0;
            return;
        }
        st->alpha = t[0] / t[1];
        st->pq_prev = t[1];
        st->first = 0;
    });
}

// x += alpha p, r -= alpha q, rr = r.r; convergence, stall -> fallback to plain CG
__global__ void __launch_bounds__(NT) k_fcg_update(float* __restrict__ x, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   size_t n, FcgState* st, double* partials)
{
    if (st->done) return;
    const float alpha = (float)st->alpha;
    FSum acc;
    GRID_STRIDE(i, n)
    {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float rv = fmaf(-alpha, q[i], r[i]);
        r[i] = rv;
        acc.add(rv * rv);
    }
    double v1[1] = {acc.value()};
    reduce_then<1>(v1, partials, &st->counter, [&](double* t) {
        const double rr = t[0];
        st->iter += 1;
        st->rr = rr;
        st->zscale = sqrt(rr);
        if (!isfinite(rr)) { st->done = 1; st->status = -5; return; }
        if (rr <= st->tol2 * st->bb) { st->done = 1; st->status = 0; return; }
        if (st->iter >= st->max_iter) { st->done = 1; st->status = 1; return; }
        if (rr < 0.98 * st->best_rr) { st->best_rr = rr; st->since_best = 0; }
        else if (++st->since_best >= st->stall_window) {
            if (!st->use_r) {   // the network stalls: continue as plain CG
                st->use_r = 1;
                st->fallback_iter = st->iter;
                st->since_best = 0;
                st->best_rr = rr;
            } else if (st->stall_window > 0 && st->since_best >= 4 * st->stall_window) {
                st->done = 1;
                st->status = 2;
            }
        }
    });
}

int grid_n(size_t n)
{
    size_t b = (n + 4 * NT - 1) / (4 * NT);
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

int ffail(int code, const char* msg) { return bsk::set_error(code, msg); }

#define FCUDA(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ffail(BSK_ECUDA, #call " failed");   \
    } while (0)

}  // namespace

namespace bsk {

// Inner FCG solve of A x = b (FP32) from x = 0 on the caller's work vectors. op applies
// q = A p on the handle; net maps rn to zn. Returns the FCG status; iterations and the
// fallback iteration are written to *iters and *fallback_iter.
int fcg_inner(const FcgVectors& V, size_t n, const uint8_t* mask, double tol, int max_iter, int stall_window,
              double out_scale, double jac, const std::function<int(const float*, float*)>& op, bsk_net* net,
              const std::function<int(bsk_net*, const float*, const uint8_t*, float*)>& net_forward,
              cudaStream_t s, int* iters, int* fallback_iter, int* rejected, double time_limit,
              std::chrono::steady_clock::time_point t0)
{
    FcgState* st = reinterpret_cast<FcgState*>(V.state);
    FcgState h;
    memset(&h, 0, sizeof h);
    h.tol2 = tol * tol;
    h.max_iter = max_iter;
    h.stall_window = stall_window > 0 ? stall_window : 8;
    h.use_r = net ? 0 : 1;
    const bool lin = net && net_linear(net);
    h.unit_input = lin ? 1 : 0;
    h.fallback_iter = -1;
    h.out_scale = out_scale;
    h.jac = jac;
    FCUDA(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, s));
    FCUDA(cudaStreamSynchronize(s));   // h is a stack copy
    const int gb = grid_n(n);
    k_fcg_init<<<gb, NT, 0, s>>>(V.b, V.r, V.x, n, mask, st, V.partials);
    FCUDA(cudaGetLastError());
    FCUDA(cudaMemsetAsync(V.q, 0, n * sizeof(float), s));
    FCUDA(cudaMemsetAsync(V.p, 0, n * sizeof(float), s));
    int k = 0;
    for (;;) {
        // a few iterations between polls
        for (int j = 0; j < 4; j++, k++) {
            if (V.rec_r && k < V.rec_steps) {   // the state this iteration starts from
                FCUDA(cudaMemcpyAsync(V.rec_r + (size_t)k * n, V.r, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
                FCUDA(cudaMemcpyAsync(V.rec_x + (size_t)k * n, V.x, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
            }
            if (net) {
                if (!lin) {
                    k_fcg_normalise<<<gb, NT, 0, s>>>(V.r, V.rn, n, st);
                    FCUDA(cudaGetLastError());
                }
                if (int rc = net_forward(net, lin ? V.r : V.rn, mask, V.zn)) return rc;
            }
            k_fcg_direction<<<gb, NT, 0, s>>>(net ? V.zn : V.r, V.z, V.r, V.q, n, st, V.partials);
            k_fcg_p<<<gb, NT, 0, s>>>(V.z, V.r, V.p, n, st);
            FCUDA(cudaGetLastError());
            if (int rc = op(V.p, V.q)) return rc;
            k_fcg_alpha<<<gb, NT, 0, s>>>(V.r, V.p, V.q, n, st, V.partials);
            k_fcg_update<<<gb, NT, 0, s>>>(V.x, V.r, V.p, V.q, n, st, V.partials);
            FCUDA(cudaGetLastError());
        }
        FCUDA(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s));
        FCUDA(cudaStreamSynchronize(s));
        if (h.done) break;
        if (time_limit > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > time_limit)
            return ffail(BSK_ETIMEOUT, "FCG exceeded its time limit");
    }
    *iters = h.iter;
    *fallback_iter = h.fallback_iter;
    *rejected = h.rejected;
    switch (h.status) {
    case 0: return BSK_OK;
    case 1: return BSK_NOT_CONVERGED;
    case 2: return BSK_STALLED;
    default: return ffail(BSK_EBREAKDOWN, "FCG breakdown (p.Ap <= 0 or non-finite)");
    }
}

size_t fcg_state_bytes() { return sizeof(FcgState); }

}  // namespace bsk
