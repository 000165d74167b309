// bsk_api.cu -- the C ABI declared in include/bsk.h: kernel tables, solver handles, the CG
// loop (device-resident iteration in CUDA graphs, host polling), iterative refinement,
// implicit Euler stepping, boundary and preconditioner set-up and the coarse-to-fine
// prolongation. Every arithmetic step of the path runs in the library's kernels; this file
// computes the small host tables (kernels, band rows, quadrature), validates, allocates and
// sequences.
#include <algorithm>
#include <vector>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>

#include "bsk.h"
#include "bsk_launch.h"
#include "host_bspline.h"

using bsk::Scalars;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(BSK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BSK_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
    } while (0)

// m! * beta^m(j) for odd m: with (m+1)/2 an integer every term of the truncated-power sum
// (beta^m = (m+1)-fold convolution of the unit box, Table tblBsplines) is an integer, so the
// value is exact in 64-bit arithmetic for m <= 11.
long long bspline_odd_scaled(int m, int j)
{
    const int half = (m + 1) / 2;
    long long s = 0, binom = 1;
    for (int k = 0; k <= m + 1; k++) {
        long long t = (long long)j + half - k;
        if (t > 0) {
            long long p = 1;
            for (int e = 0; e < m; e++) p *= t;
            s += (k & 1) ? -binom * p : binom * p;
        }
        binom = binom * (m + 1 - k) / (k + 1);
    }
    return s;
}

// beta^m(j) at an integer j, exactly: m! 2^m beta^m(j) = sum_k (-1)^k C(m+1, k) (2j + m + 1 - 2k)_+^m
// (the truncated-power form with every term an integer, for either parity of m).
double bspline_at(int m, int j)
{
    long long s = 0, binom = 1;
    for (int k = 0; k <= m + 1; k++) {
        const long long t = 2LL * j + m + 1 - 2LL * k;
        if (t > 0) {
            long long pw = 1;
            for (int e = 0; e < m; e++) pw *= t;
            s += (k & 1) ? -binom * pw : binom * pw;
        }
        binom = binom * (m + 1 - k) / (k + 1);
    }
    double den = 1.0;
    for (int i = 2; i <= m; i++) den *= i;
    return (double)s / (den * (double)(1LL << m));
}

double factorial(int m)
{
    double f = 1.0;
    for (int i = 2; i <= m; i++) f *= i;
    return f;
}

}  // namespace

extern "C" int bspline_kernels(int n, double h, double* mass, double* stiff)
{
    if (n < 1 || n > 5) return fail(BSK_EINVAL, "degree %d outside 1..5", n);
    if (!(h > 0.0) || !std::isfinite(h)) return fail(BSK_EINVAL, "grid step must be > 0");
    if (!mass || !stiff) return fail(BSK_EINVAL, "null output array");
    // scalar-product row of Table tblBsplines: integral beta^n(x-k) beta^n(x-l) = beta^{2n+1}(k-l);
    // with the derivative row, integral beta^n'(x-k) beta^n'(x-l) = -(second difference of
    // beta^{2n-1}) at k-l.
    const int mm = 2 * n + 1, mk = 2 * n - 1;
    const double fm = factorial(mm), fk = factorial(mk);
    for (int j = -n; j <= n; j++) {
        const double m1 = (double)bspline_odd_scaled(mm, j) / fm;
        const long long d2 = bspline_odd_scaled(mk, j + 1) - 2 * bspline_odd_scaled(mk, j) +
                             bspline_odd_scaled(mk, j - 1);
        const double k1 = -(double)d2 / fk;
        mass[j + n] = h * m1;
        stiff[j + n] = k1 / h;
    }
    return BSK_OK;
}

struct bsk_handle {
    int nx, ny, nz, n, prec;
    double h[3];
    double dt;
    size_t len;
    cudaStream_t stream;       // the caller's stream: every launch goes here
    cudaStream_t cap_stream;   // private stream used only to capture the CG graph (the legacy
                               // default stream cannot be captured; the graph runs on `stream`)
    uint8_t* mask;
    uint32_t* mbits;              // the mask bit-packed for the TMA kernels (TMA grids), or null
    uint8_t* occ;                 // tile occupancy per plane of the mask (TMA grids), or null
    double M[3][bsk::kMaxTaps];   // per-axis mass kernels
    double K[3][bsk::kMaxTaps];   // per-axis stiffness kernels (not yet multiplied by dt)
    // CG vectors in the CG element type (double for BSK_F64, float otherwise). The single-pass
    // TMA iteration ping-pongs r, q and p (r/r2, q/q2, p0/p1); the general one uses r, q, p0/p1.
    void *x, *r, *p0, *p1, *q, *bvec, *r2, *q2;
    bool use_tma;     // CG vectors go through the TMA kernels (16-byte rows; a mask only zeroes
                      // outputs, the solvers' vectors being zero on inactive nodes)
    bool tma64;       // FP64 operator passes (op_apply / residual) may use the TMA kernels
    bool res_df;      // BSK_F32_IR: the true residual may use the double-float TMA kernel
    // iterative refinement (FP64 outer vectors)
    double *r64, *b64;
    Scalars *sc, *sc64, *sc_aux;
    Scalars* h_sc;   // pinned host mirror
    double* partials;
    unsigned int* work;   // item-queue counters of the TMA kernels
    cudaGraphExec_t graph;
    int graph_chunk;
    long long launches;   // kernels launched since the counter was last read
    cudaEvent_t it_ev[2]; // bracket the inner iterations on `stream` (bsk_cg_report.iter_ms)
    double iter_ms;       // device time of the inner iterations since the counter was last read
    void* tr_L[3];        // Cholesky factors of the sampled basis per axis (first direct transform)
    // variable coefficients (bsk_set_coefficients): D and mu_a at the (nz+2)(ny+2)(nx+2) nodes as
    // float [0] (FP32 passes) and double [1] (FP64 passes); null = constant coefficients
    void* cd[2];
    void* cm[2];
    bool use_tma0, tma640, res_df0;   // TMA eligibility of the constant-coefficient operator
    int cg_impl;          // single-pass FP32 CG iteration: 0 = warp-specialised, 1 = op_tma.cuh
    int ws_chunk;         // warp-specialised CG pass: most planes per z-chunk (0 = its default)
    int bc;               // BSK_BC_DIRICHLET (odd reflection) or BSK_BC_ROBIN (untruncated basis)
    double pen;           // Robin: weight of the boundary term
    void* rb[2];          // Robin: band rows near the faces, float [0] / double [1]
    int pc;               // BSK_PC_NONE or BSK_PC_JACOBI
    void* jac[2];         // Jacobi: per-axis diagonals [3][2][jn], float [0] / double [1]
    int jn;
    void* jvec;           // Jacobi: 1 / diag A per node, CG precision
    float* fcg_ws;        // FCG work vectors z, rn, zn (allocated by the first fcg_solve)
    double* fcg_partials;
    void* fcg_state;
    // z-slab placement (bsk_set_slab): global offset and plane count (0 = not a slab), and the
    // reduction scratch of the slab CG passes
    int z_off, nz_glob;
    double* slab_partials;
    unsigned* slab_ctr;
    // heat_step_host: device copies of the caller's host u and q (allocated by the first call)
    void *u_dev, *q_dev;
    cudaEvent_t io_ev[4];
};

namespace {

size_t user_es(const bsk_handle* h)
{
    return h->prec == BSK_BF16S ? 2 : h->prec == BSK_F32 ? sizeof(float) : sizeof(double);
}
size_t cg_es(const bsk_handle* h) { return h->prec == BSK_F64 ? sizeof(double) : sizeof(float); }

void fill_tma(const bsk_handle* h, bsk::TmaLaunch& L, int mode)
{
    memset(&L, 0, sizeof L);
    L.work = h->work;
    L.mode = mode;
    L.impl = h->cg_impl;
    L.ws_chunk = h->ws_chunk;
    L.degree = h->n;
    L.nx = h->nx;
    L.ny = h->ny;
    L.nz = h->nz;
    L.mask = h->mask;
    L.mbits = h->mbits;
    L.occ = h->occ;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < bsk::kMaxTaps; j++) {
            L.M[d][j] = h->M[d][j];
            L.Kdt[d][j] = h->dt * h->K[d][j];
        }
}

// Vectors of single-pass CG pass `it` (op_tma.cuh / op_ws.cuh). The pass keeps no r: it reads
// p_{m-1}, q_{m-1} and p_{m-2} and writes p_m and q_m, so p and q each rotate through three
// buffers (period 3; pass 0 reads r_0 from h->r as "p_{-1}", with p_{-2} = h->p0 and q = h->q
// zero). Graph chunks are multiples of 3 so that every launch starts from the same buffers.
void cg1_vectors(const bsk_handle* h, int it, bsk::TmaLaunch& L)
{
    void* P[3] = {h->r, h->p1, h->p0};
    void* Q[3] = {h->q, h->q2, h->r2};
    const int i = it % 3, o = (it + 1) % 3, older = (it + 2) % 3;
    L.in[0] = P[i];
    L.in[1] = Q[i];
    L.in[2] = P[older];
    L.inint = h->x;
    L.out0 = Q[o];
    L.out1 = nullptr;
    L.out2 = P[o];
    L.xvec = h->x;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// May a pass of element size es over these vectors use the TMA kernels?
bool tma_ok(const bsk_handle* h, size_t es, std::initializer_list<const void*> ptrs)
{
    const bool allowed = es == sizeof(double) ? h->tma64 : h->use_tma;
    if (!allowed) return false;
    for (const void* p : ptrs)
        if (!aligned16(p)) return false;
    return true;
}

// Can the single-pass FP32 CG iteration of this handle run as the warp-specialised pass?
bool cg_ws_eligible(const bsk_handle* h)
{
    return h->use_tma0 && (h->prec == BSK_F32 || h->prec == BSK_F32_IR) && !h->mask && bsk::ws_supported(h->n);
}

cudaError_t tma_launch_es(size_t es, const bsk::TmaLaunch& L, cudaStream_t s)
{
    return es == sizeof(double) ? bsk::launch_tma<double>(L, s) : bsk::launch_tma<float>(L, s);
}

void fill_launch(const bsk_handle* h, bsk::OpLaunch& L, int mode)
{
    memset(&L, 0, sizeof L);
    L.mode = mode;
    L.degree = h->n;
    L.nx = h->nx;
    L.ny = h->ny;
    L.nz = h->nz;
    L.mask = h->mask;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < bsk::kMaxTaps; j++) {
            L.M[d][j] = h->M[d][j];
            L.Kdt[d][j] = h->dt * h->K[d][j];
        }
    for (int i = 0; i < 2; i++) {
        L.vd[i] = h->cd[i];
        L.vm[i] = h->cm[i];
    }
    for (int d = 0; d < 3; d++) L.h[d] = h->h[d];
    L.dt = h->dt;
    for (int i = 0; i < 2; i++) {
        L.rb[i] = h->bc == BSK_BC_ROBIN ? h->rb[i] : nullptr;
        L.jac[i] = h->pc && !h->jvec ? h->jac[i] : nullptr;
        L.jvec[i] = h->pc && (cg_es(h) == sizeof(double)) == (i == 1) ? h->jvec : nullptr;
    }
    L.jn = h->jn;
}

template <typename T>
cudaError_t op_launch(const bsk::OpLaunch& L, cudaStream_t s)
{
    return bsk::launch_op<T>(L, s);
}

cudaError_t op_launch_es(size_t es, const bsk::OpLaunch& L, cudaStream_t s)
{
    return es == sizeof(double) ? bsk::launch_op<double>(L, s) : bsk::launch_op<float>(L, s);
}

// Counts one kernel launch of the handle (for the launch totals of bsk_cg_report).
#define BSK_LAUNCH(h, call)          \
    do {                             \
        BSK_CUDA(call);              \
        (h)->launches += 1;          \
    } while (0)

int sync_scalars(bsk_handle* h, Scalars* dev)
{
    BSK_CUDA(cudaMemcpyAsync(h->h_sc, dev, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    return BSK_OK;
}

int init_scalars(bsk_handle* h, Scalars* dev, double tol, int max_iter, int stall_window)
{
    Scalars s;
    memset(&s, 0, sizeof s);
    s.tol2 = tol * tol;
    s.max_iter = max_iter;
    s.stall_window = stall_window;
    s.pc = h->pc != BSK_PC_NONE;
    // the pinned mirror is reused as the staging buffer: wait for earlier copies out of it
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    *h->h_sc = s;
    BSK_CUDA(cudaMemcpyAsync(dev, h->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, h->stream));
    // a kernel stopped by a wait time-out may have left the item-queue counters non-zero
    BSK_CUDA(cudaMemsetAsync(h->work, 0, 2 * sizeof(unsigned int), h->stream));
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    return BSK_OK;
}

struct Opts {
    double tol, inner_tol, time_limit;
    int max_iter, check_every, stall_window, max_outer, residual_fp64;
};

Opts resolve(const bsk_cg_opts* o)
{
    Opts r;
    r.tol = (o && o->tol > 0) ? o->tol : 1e-8;
    r.max_iter = (o && o->max_iter > 0) ? o->max_iter : 10000;
    r.check_every = (o && o->check_every > 0) ? o->check_every : 16;
    // a multiple of 6: the two-pass iteration's p alternates between two buffers and the
    // single-pass iteration's p and q rotate through three, and each graph launch must start
    // from the same buffers
    r.check_every = (r.check_every + 5) / 6 * 6;
    r.stall_window = (o && o->stall_window > 0) ? o->stall_window : 0;
    r.inner_tol = (o && o->inner_tol > 0) ? o->inner_tol : 1e-5;
    r.max_outer = (o && o->max_outer > 0) ? o->max_outer : 30;
    r.time_limit = (o && o->time_limit_s > 0) ? o->time_limit_s : 0.0;
    r.residual_fp64 = (o && o->residual_fp64) ? 1 : 0;
    return r;
}

// Enqueues the true residual r = b - A x of FP64 vectors (FIN_RES_TRUE: r.r and b.b into sc):
// double-float TMA kernel (BSK_F32_IR, unless fp64), FP64 TMA kernel, or the general kernel.
int enqueue_residual64(bsk_handle* h, const double* b, const double* x, double* r, Scalars* sc, bool fp64)
{
    if (tma_ok(h, sizeof(double), {b, x, r})) {
        bsk::TmaLaunch R;
        fill_tma(h, R, bsk::TMODE_RES);
        R.in[0] = x;
        R.inint = b;
        R.out0 = r;
        R.sc = sc;
        R.partials = h->partials;
        R.fin = bsk::FIN_RES_TRUE;
        if (h->res_df && !fp64) BSK_LAUNCH(h, bsk::launch_tma<bsk::dfl>(R, h->stream));
        else BSK_LAUNCH(h, bsk::launch_tma<double>(R, h->stream));
    } else {
        bsk::OpLaunch L;
        fill_launch(h, L, bsk::MODE_RES);
        L.in0 = x;
        L.b = b;
        L.out0 = r;
        L.sc = sc;
        L.partials = h->partials;
        L.fin = bsk::FIN_RES_TRUE;
        BSK_LAUNCH(h, op_launch<double>(L, h->stream));
    }
    return BSK_OK;
}

// The device-resident CG chunk: `chunk` iterations of (fused p-update + operator + p.Ap, then
// r update + r.r), captured once per handle into a CUDA graph and replayed.
template <typename T>
int enqueue_chunk(bsk_handle* h, int chunk)
{
    cudaStream_t s = h->cap_stream;
    T* p[2] = {static_cast<T*>(h->p0), static_cast<T*>(h->p1)};
    if (h->use_tma) {
        // one kernel per iteration: pass m reads p_{m-1}, q_{m-1}, p_{m-2} and writes p_m, q_m
        for (int it = 0; it < chunk; it++) {
            bsk::TmaLaunch L;
            fill_tma(h, L, bsk::TMODE_CG);
            cg1_vectors(h, it, L);
            L.sc = h->sc;
            L.partials = h->partials;
            L.fin = bsk::FIN_CG1;
            BSK_CUDA(bsk::launch_tma<T>(L, s));
        }
        return BSK_OK;
    }
    for (int it = 0; it < chunk; it++) {
        bsk::OpLaunch L;
        fill_launch(h, L, bsk::MODE_CGP);
        L.in0 = h->r;
        L.in1 = p[it & 1];
        L.out0 = h->q;
        L.out1 = p[(it + 1) & 1];
        L.xvec = h->x;
        L.sc = h->sc;
        L.partials = h->partials;
        L.fin = bsk::FIN_CGP;
        L.p_parity = (it + 1) & 1;
        BSK_CUDA(op_launch<T>(L, s));
        if (h->pc)
            BSK_CUDA(bsk::launch_cg_update_pc<T>(static_cast<T*>(h->r), static_cast<const T*>(h->q), h->len,
                                                 h->nx, h->ny, static_cast<const T*>(h->jac[sizeof(T) == 8]),
                                                 h->jn, static_cast<const T*>(h->jvec), h->sc, h->partials,
                                                 bsk::FIN_UPD_PC, s));
        else
            BSK_CUDA(bsk::launch_cg_update<T>(static_cast<T*>(h->r), static_cast<const T*>(h->q),
                                              h->len, h->sc, h->partials, bsk::FIN_UPD, s));
    }
    return BSK_OK;
}

// Preconditioned CG: r.z of the starting residual (after the init kernel has set r and rr).
template <typename T>
int pc_start(bsk_handle* h)
{
    if (!h->pc) return BSK_OK;
    BSK_LAUNCH(h, bsk::launch_pc_dot<T>(static_cast<const T*>(h->r), h->len, h->nx, h->ny,
                                        static_cast<const T*>(h->jac[sizeof(T) == 8]), h->jn,
                                        static_cast<const T*>(h->jvec), h->sc, h->partials, h->stream));
    return BSK_OK;
}

template <typename T>
int ensure_graph(bsk_handle* h, int chunk)
{
    if (h->graph && h->graph_chunk == chunk) return BSK_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    BSK_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_chunk<T>(h, chunk);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != BSK_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_chunk = chunk;
    return BSK_OK;
}

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Runs the CG iteration on the handle's CG vectors from the state set up by an init kernel
// (r, rr, bb in h->sc; p0 zeroed), until the device reports done. Returns the CG status.
template <typename T>
int run_iterations(bsk_handle* h, const Opts& o, std::chrono::steady_clock::time_point t0,
                   int* iters_out)
{
    int rc = ensure_graph<T>(h, o.check_every);
    if (rc) return rc;
    if ((rc = sync_scalars(h, h->sc))) return rc;
    BSK_CUDA(cudaEventRecord(h->it_ev[0], h->stream));
    while (!h->h_sc->done) {
        BSK_CUDA(cudaGraphLaunch(h->graph, h->stream));
        h->launches += (h->use_tma ? 1LL : 2LL) * h->graph_chunk;
        if ((rc = sync_scalars(h, h->sc))) return rc;
        if (o.time_limit > 0 && !h->h_sc->done && seconds_since(t0) > o.time_limit) {
            *iters_out = h->h_sc->iter;
            return fail(BSK_ETIMEOUT, "solve exceeded its time limit of %.3f s", o.time_limit);
        }
    }
    BSK_CUDA(cudaEventRecord(h->it_ev[1], h->stream));
    BSK_CUDA(cudaEventSynchronize(h->it_ev[1]));
    float ms = 0.f;
    BSK_CUDA(cudaEventElapsedTime(&ms, h->it_ev[0], h->it_ev[1]));
    h->iter_ms += ms;
    if (!h->use_tma)   // the single-pass iteration leaves no x update pending
        BSK_LAUNCH(h, bsk::launch_cg_flush<T>(static_cast<T*>(h->x), static_cast<const T*>(h->p0),
                                         static_cast<const T*>(h->p1), h->len, h->sc, h->stream));
    *iters_out = h->h_sc->iter;
    switch (h->h_sc->status) {
    case 0: return BSK_OK;
    case 1: return BSK_NOT_CONVERGED;
    case 2: return BSK_STALLED;
    default: return fail(BSK_EBREAKDOWN, "CG breakdown (p.Ap <= 0 or non-finite reduction)");
    }
}

// Plain CG (BSK_F64 / BSK_F32): x (user) is copied into the handle's x, solved, copied back.
template <typename T>
int cg_plain(bsk_handle* h, const T* b, T* x, const Opts& o, bsk_cg_report* rep,
             std::chrono::steady_clock::time_point t0)
{
    int rc;
    BSK_LAUNCH(h, bsk::launch_copy_masked<T>(x, static_cast<T*>(h->x), h->len, h->mask, h->stream));
    if ((rc = init_scalars(h, h->sc, o.tol, o.max_iter, o.stall_window))) return rc;
    bsk::OpLaunch L;
    if (tma_ok(h, sizeof(T), {b})) {
        bsk::TmaLaunch R;
        fill_tma(h, R, bsk::TMODE_RES);
        R.in[0] = h->x;
        R.inint = b;
        R.out0 = h->r;
        R.sc = h->sc;
        R.partials = h->partials;
        R.fin = bsk::FIN_RES_INIT;
        BSK_LAUNCH(h, bsk::launch_tma<T>(R, h->stream));
    } else {
        fill_launch(h, L, bsk::MODE_RES);
        L.in0 = h->x;
        L.b = b;
        L.out0 = h->r;
        L.sc = h->sc;
        L.partials = h->partials;
        L.fin = bsk::FIN_RES_INIT;
        BSK_LAUNCH(h, op_launch<T>(L, h->stream));
    }
    if ((rc = pc_start<T>(h))) return rc;
    BSK_CUDA(cudaMemsetAsync(h->p0, 0, h->len * sizeof(T), h->stream));
    if (h->use_tma) BSK_CUDA(cudaMemsetAsync(h->q, 0, h->len * sizeof(T), h->stream));
    int iters = 0;
    int st = run_iterations<T>(h, o, t0, &iters);
    if (st < 0 && st != BSK_EBREAKDOWN) return st;
    if (h->h_sc->zero_b) BSK_CUDA(cudaMemsetAsync(h->x, 0, h->len * sizeof(T), h->stream));
    BSK_LAUNCH(h, bsk::launch_copy_masked<T>(static_cast<const T*>(h->x), x, h->len, h->mask, h->stream));
    // true residual of the returned x
    if (tma_ok(h, sizeof(T), {b, x})) {
        bsk::TmaLaunch R;
        fill_tma(h, R, bsk::TMODE_RES);
        R.in[0] = x;
        R.inint = b;
        R.out0 = h->r;
        R.sc = h->sc_aux;
        R.partials = h->partials;
        R.fin = bsk::FIN_RES_TRUE;
        BSK_LAUNCH(h, bsk::launch_tma<T>(R, h->stream));
    } else {
        fill_launch(h, L, bsk::MODE_RES);
        L.in0 = x;
        L.b = b;
        L.out0 = h->r;
        L.sc = h->sc_aux;
        L.partials = h->partials;
        L.fin = bsk::FIN_RES_TRUE;
        BSK_LAUNCH(h, op_launch<T>(L, h->stream));
    }
    if ((rc = sync_scalars(h, h->sc_aux))) return rc;
    if (rep) {
        rep->iterations += iters;
        rep->rel_residual = h->h_sc->bb_true > 0 ? std::sqrt(h->h_sc->rr_true / h->h_sc->bb_true) : 0.0;
    }
    return st;
}

// Mixed precision: FP64 true residual and update around inner FP32 CG solves.
int cg_ir(bsk_handle* h, const double* b, double* x, const Opts& o, bsk_cg_report* rep,
          std::chrono::steady_clock::time_point t0)
{
    int rc;
    int total_iters = 0, outer = 0, st = BSK_NOT_CONVERGED;
    double rel = 0.0;
    BSK_LAUNCH(h, bsk::launch_copy_masked<double>(x, x, h->len, h->mask, h->stream));
    for (;; outer++) {
        if ((rc = enqueue_residual64(h, b, x, h->r64, h->sc64, o.residual_fp64))) return rc;
        if ((rc = sync_scalars(h, h->sc64))) return rc;
        const double rr = h->h_sc->rr_true, bb = h->h_sc->bb_true;
        if (!std::isfinite(rr) || !std::isfinite(bb))
            return fail(BSK_EBREAKDOWN, "non-finite residual in iterative refinement");
        if (bb == 0.0) {
            BSK_CUDA(cudaMemsetAsync(x, 0, h->len * sizeof(double), h->stream));
            rel = 0.0;
            st = BSK_OK;
            break;
        }
        rel = std::sqrt(rr / bb);
        if (rel <= o.tol) { st = BSK_OK; break; }
        if (outer >= o.max_outer || total_iters >= o.max_iter) { st = BSK_NOT_CONVERGED; break; }
        if (o.time_limit > 0 && seconds_since(t0) > o.time_limit) {
            if (rep) { rep->iterations += total_iters; rep->outer_iterations += outer; rep->rel_residual = rel; }
            return fail(BSK_ETIMEOUT, "solve exceeded its time limit of %.3f s", o.time_limit);
        }
        // inner FP32 solve of A d = r / ||r|| from d = 0, only as accurately as this step needs
        double inner = std::max(o.inner_tol, 0.3 * o.tol / rel);
        if (inner > 0.5) inner = 0.5;
        BSK_LAUNCH(h, bsk::launch_ir_scale_down(h->r64, static_cast<float*>(h->r), h->len, h->sc64,
                                           h->stream));
        if ((rc = init_scalars(h, h->sc, inner, o.max_iter - total_iters, o.stall_window))) return rc;
        BSK_LAUNCH(h, bsk::launch_cg_init_zero<float>(static_cast<const float*>(h->r),
                                                 static_cast<float*>(h->r), static_cast<float*>(h->x),
                                                 h->len, h->mask, h->sc, h->partials, h->stream));
        if ((rc = pc_start<float>(h))) return rc;
        BSK_CUDA(cudaMemsetAsync(h->p0, 0, h->len * sizeof(float), h->stream));
        if (h->use_tma) BSK_CUDA(cudaMemsetAsync(h->q, 0, h->len * sizeof(float), h->stream));
        int it = 0;
        int ist = run_iterations<float>(h, o, t0, &it);
        total_iters += it;
        if (ist == BSK_ETIMEOUT) {
            if (rep) { rep->iterations += total_iters; rep->outer_iterations += outer + 1; rep->rel_residual = rel; }
            return ist;
        }
        if (ist < 0 && ist != BSK_EBREAKDOWN) return ist;
        if (ist == BSK_EBREAKDOWN && it == 0) return ist;
        BSK_LAUNCH(h, bsk::launch_ir_update(x, static_cast<const float*>(h->x), h->len, h->sc64, h->stream));
    }
    if (rep) {
        rep->iterations += total_iters;
        rep->outer_iterations += outer;
        rep->rel_residual = rel;
    }
    return st;
}

int check_handle(const bsk_handle* h)
{
    if (!h) return fail(BSK_EINVAL, "null handle");
    return BSK_OK;
}

int solve_dispatch(bsk_handle* h, const void* b, void* x, const Opts& o, bsk_cg_report* rep,
                   std::chrono::steady_clock::time_point t0)
{
    switch (h->prec) {
    case BSK_F64: return cg_plain<double>(h, (const double*)b, (double*)x, o, rep, t0);
    case BSK_F32: return cg_plain<float>(h, (const float*)b, (float*)x, o, rep, t0);
    default: return cg_ir(h, (const double*)b, (double*)x, o, rep, t0);
    }
}

bool overlaps(const void* a, const void* b, size_t bytes)
{
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + bytes && pb < pa + bytes;
}

}  // namespace

extern "C" int bsk_create(const bsk_problem* prob, int precision, void* stream, bsk_handle** out)
{
    if (!prob || !out) return fail(BSK_EINVAL, "null argument");
    *out = nullptr;
    const int n = prob->degree;
    if (n < 1 || n > 5) return fail(BSK_EINVAL, "degree %d outside 1..5", n);
    if (prob->nx < n || prob->ny < n || prob->nz < n)
        return fail(BSK_EINVAL, "each axis needs at least degree (%d) unknowns, got %d x %d x %d", n,
                    prob->nx, prob->ny, prob->nz);
    if (!(prob->hx > 0) || !(prob->hy > 0) || !(prob->hz > 0) || !std::isfinite(prob->hx) ||
        !std::isfinite(prob->hy) || !std::isfinite(prob->hz))
        return fail(BSK_EINVAL, "grid steps must be finite and > 0");
    if (!(prob->dt >= 0) || !std::isfinite(prob->dt)) return fail(BSK_EINVAL, "dt must be finite and >= 0");
    if (precision != BSK_F64 && precision != BSK_F32 && precision != BSK_F32_IR && precision != BSK_BF16S)
        return fail(BSK_EINVAL, "unknown precision %d", precision);
    const size_t len = (size_t)prob->nx * prob->ny * prob->nz;
    if ((size_t)prob->nx * prob->ny > (size_t)1 << 31 || len > ((size_t)1 << 40))
        return fail(BSK_EINVAL, "grid too large");

    bsk_handle* h = new (std::nothrow) bsk_handle;
    if (!h) return fail(BSK_ENOMEM, "host allocation failed");
    memset(h, 0, sizeof *h);
    h->nx = prob->nx;
    h->ny = prob->ny;
    h->nz = prob->nz;
    h->n = n;
    h->prec = precision;
    h->h[0] = prob->hx;
    h->h[1] = prob->hy;
    h->h[2] = prob->hz;
    h->dt = prob->dt;
    h->len = len;
    h->stream = (cudaStream_t)stream;
    for (int d = 0; d < 3; d++) {
        double m[bsk::kMaxTaps] = {0}, k[bsk::kMaxTaps] = {0};
        bspline_kernels(n, h->h[d], m, k);
        for (int j = 0; j < 2 * n + 1; j++) {
            h->M[d][j] = m[j];
            h->K[d][j] = k[j];
        }
    }
    auto cleanup = [&](int code) {
        bsk_destroy(h);
        return code;
    };
    cudaError_t e;
#define BSK_ALLOC(ptr, bytes)                                                                  \
    do {                                                                                       \
        e = cudaMalloc((void**)&(ptr), (bytes));                                               \
        if (e != cudaSuccess) {                                                                \
            cudaGetLastError();                                                                \
            int c_ = fail(e == cudaErrorMemoryAllocation ? BSK_ENOMEM : BSK_ECUDA,             \
                          "cudaMalloc(%zu) failed: %s", (size_t)(bytes), cudaGetErrorString(e)); \
            bsk_destroy(h);                                                                    \
            return c_;                                                                         \
        }                                                                                      \
    } while (0)

    e = bsk::prepare_op<float>(n);
    if (e == cudaSuccess) e = bsk::prepare_op<double>(n);
    if (e == cudaSuccess) e = bsk::prepare_var<float>(n);
    if (e == cudaSuccess) e = bsk::prepare_var<double>(n);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "kernel set-up"));
    {
        // the TMA kernels need grids whose rows are whole 16-byte units
        const size_t ces_ = precision == BSK_F64 ? sizeof(double) : sizeof(float);
        h->use_tma = n <= (ces_ == 8 ? bsk::tma_max_degree<double>() : bsk::tma_max_degree<float>()) &&
                     (prob->nx * ces_) % 16 == 0 && precision != BSK_BF16S;
        h->tma64 = n <= bsk::tma_max_degree<double>() && (prob->nx * sizeof(double)) % 16 == 0 &&
                   precision != BSK_F32 && precision != BSK_BF16S;
        if (h->use_tma || precision == BSK_F32) {
            e = bsk::prepare_tma<float>(n > bsk::tma_max_degree<float>() ? 1 : n);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "TMA kernel set-up"));
        }
        if (h->tma64 || (h->use_tma && ces_ == 8)) {
            e = bsk::prepare_tma<double>(n);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "TMA kernel set-up"));
        }
        h->res_df = precision == BSK_F32_IR && h->tma64 && n <= bsk::tma_max_degree<bsk::dfl>();
        if (h->res_df) {
            e = bsk::prepare_tma<bsk::dfl>(n);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "TMA kernel set-up"));
        }
        h->use_tma0 = h->use_tma;
        h->tma640 = h->tma64;
        h->res_df0 = h->res_df;
    }
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    for (int i = 0; i < 2; i++) {
        e = cudaEventCreate(&h->it_ev[i]);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaEventCreate"));
    }
    if (prob->mask) {
        BSK_ALLOC(h->mask, len);
        e = cudaMemcpyAsync(h->mask, prob->mask, len, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "mask copy"));
        if (h->use_tma || h->tma64) {
            // brick occupancy of the mask: the TMA kernels skip the (tile, z-chunk) items that
            // hold no active node
            BSK_ALLOC(h->occ, (size_t)bsk::tma_tiles(prob->nx, prob->ny) * prob->nz);
            e = bsk::launch_tile_occupancy(h->mask, prob->nx, prob->ny, prob->nz, h->occ, h->stream);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "occupancy launch"));
            // and the mask itself as bits, which the TMA kernels read (1/8 byte per unknown)
            BSK_ALLOC(h->mbits, (size_t)bsk::mask_words(prob->nx) * prob->ny * prob->nz * sizeof(uint32_t));
            e = bsk::launch_pack_mask(h->mask, prob->nx, prob->ny, prob->nz, h->mbits, h->stream);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "mask packing launch"));
        }
    }
    const size_t ces = cg_es(h);
    if (precision != BSK_BF16S) {   // the BF16-storage variant has no solver
        BSK_ALLOC(h->x, len * ces);
        BSK_ALLOC(h->r, len * ces);
        BSK_ALLOC(h->p0, len * ces);
        BSK_ALLOC(h->p1, len * ces);
        BSK_ALLOC(h->q, len * ces);
        if (h->use_tma) {
            BSK_ALLOC(h->r2, len * ces);
            BSK_ALLOC(h->q2, len * ces);
        }
        if (precision == BSK_F32_IR) {
            BSK_ALLOC(h->r64, len * sizeof(double));
            BSK_ALLOC(h->b64, len * sizeof(double));
        } else {
            BSK_ALLOC(h->bvec, len * ces);
        }
    }
    if (h->occ) {
        // items skipped by occupancy leave their outputs untouched: every work vector starts
        // zero, so its inactive part stays zero
        for (void* v : {h->x, h->r, h->p0, h->p1, h->q, h->r2, h->q2, h->bvec})
            if (v) {
                e = cudaMemsetAsync(v, 0, len * ces, h->stream);
                if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
            }
        for (void* v : {(void*)h->r64, (void*)h->b64})
            if (v) {
                e = cudaMemsetAsync(v, 0, len * sizeof(double), h->stream);
                if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
            }
    }
    BSK_ALLOC(h->sc, sizeof(Scalars));
    BSK_ALLOC(h->sc64, sizeof(Scalars));
    BSK_ALLOC(h->sc_aux, sizeof(Scalars));
    size_t nb = 2 * std::max(bsk::op_grid_blocks(h->nx, h->ny, h->nz, n), (size_t)bsk::vec_grid(len));
    nb = std::max(nb, 2 * bsk::var_grid_blocks<float>(h->nx, h->ny, h->nz, n));
    nb = std::max(nb, 2 * bsk::var_grid_blocks<double>(h->nx, h->ny, h->nz, n));
    for (int mode = 0; mode < 3; mode++) {
        nb = std::max(nb, 3 * (size_t)bsk::tma_grid<float>(n, mode));
        nb = std::max(nb, 3 * (size_t)bsk::tma_grid<double>(n, mode));
    }
    BSK_ALLOC(h->partials, nb * sizeof(double));
    BSK_ALLOC(h->work, 2 * sizeof(unsigned int));
    e = cudaMemsetAsync(h->work, 0, 2 * sizeof(unsigned int), h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
    e = cudaMallocHost((void**)&h->h_sc, sizeof(Scalars));
    if (e != cudaSuccess) return cleanup(fail(BSK_ENOMEM, "pinned allocation failed"));
    memset(h->h_sc, 0, sizeof(Scalars));
    for (Scalars* s : {h->sc, h->sc64, h->sc_aux}) {
        e = cudaMemsetAsync(s, 0, sizeof(Scalars), h->stream);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "bsk_create"));
#undef BSK_ALLOC
    h->cg_impl = 1;
    if (cg_ws_eligible(h)) {
        // two single-pass CG kernels implement the same iteration; neither is the faster one on
        // every grid shape, so time both on this handle's vectors and keep the faster
        if (int rc = bsk_select_cg_kernel(h, BSK_CG_KERNEL_AUTO, nullptr)) return cleanup(rc);
    }
    *out = h;
    return BSK_OK;
}

extern "C" void bsk_destroy(bsk_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    void* ptrs[] = {h->mask, h->mbits, h->occ, h->x, h->r, h->p0, h->p1, h->q, h->bvec, h->r2, h->q2, h->r64, h->b64,
                    h->sc, h->sc64, h->sc_aux, h->partials, h->work, h->cd[0], h->cd[1], h->cm[0], h->cm[1],
                    h->rb[0], h->rb[1], h->jac[0], h->jac[1], h->jvec};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_sc) cudaFreeHost(h->h_sc);
    if (h->fcg_ws) cudaFree(h->fcg_ws);
    if (h->fcg_partials) cudaFree(h->fcg_partials);
    if (h->fcg_state) cudaFree(h->fcg_state);
    if (h->slab_partials) cudaFree(h->slab_partials);
    if (h->u_dev) cudaFree(h->u_dev);
    if (h->q_dev) cudaFree(h->q_dev);
    for (int i = 0; i < 4; i++)
        if (h->io_ev[i]) cudaEventDestroy(h->io_ev[i]);
    if (h->slab_ctr) cudaFree(h->slab_ctr);
    for (int d = 0; d < 3; d++)
        if (h->tr_L[d]) cudaFree(h->tr_L[d]);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int i = 0; i < 2; i++)
        if (h->it_ev[i]) cudaEventDestroy(h->it_ev[i]);
    delete h;
}

namespace {

// Which kernels the handle may use: the TMA kernels implement the constant-coefficient operator
// with odd reflection only, and the single-pass TMA iteration has no preconditioner. Drops the
// captured CG graph (its kernels change).
void refresh_paths(bsk_handle* h)
{
    const bool plain = !h->cd[0] && !h->cd[1] && h->bc == BSK_BC_DIRICHLET;
    h->use_tma = h->use_tma0 && plain && h->pc == BSK_PC_NONE;
    h->tma64 = h->tma640 && plain;
    h->res_df = h->res_df0 && plain;
    if (h->graph) {
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

// Integral over [lo, hi] (units of h, ends on the half-integer grid) of f by (n + 1)-point Gauss
// rules on half-unit pieces: every knot of beta^n and of its integer shifts lies on that grid,
// so products of two B-splines (degree 2n) are integrated exactly.
template <typename F>
double half_unit_integral(double lo, double hi, int n, F f)
{
    if (!(hi > lo)) return 0.0;
    return bsk::host::integrate(lo, hi, (int)std::lround(2.0 * (hi - lo)), n + 1, f);
}

int dims_of(const bsk_handle* h, int ax) { return ax == 0 ? h->nx : ax == 1 ? h->ny : h->nz; }

// Robin problems: the unknowns of an axis with nt entries are the B-splines beta(x/h - i),
// i = i0 .. nt - 1 + i0 (i0 = -floor(n/2)), on the box [0, L h], L = nt - 1 + 2 i0: all those whose
// support meets the box. Band rows of the N + 1 positions nearest each face,
// [2 (mass, stiffness)][3 axes][2 ends][N + 1][2N + 1]: mass h int beta_a beta_b, stiffness
// dt / h int beta_a' beta_b' + pen (beta_a beta_b at the two faces), integrals over the box.
void robin_rows(const bsk_handle* h, std::vector<double>& out)
{
    const int n = h->n, NR = n + 1, W = 2 * n + 1, i0 = -(n / 2);
    const double s = 0.5 * (n + 1);
    out.assign((size_t)2 * 3 * 2 * NR * W, 0.0);
    auto at = [&](int m, int ax, int end, int r, int c) -> double& {
        return out[((((size_t)m * 3 + ax) * 2 + end) * NR + r) * W + c];
    };
    for (int ax = 0; ax < 3; ax++) {
        const int nt = dims_of(h, ax);
        const double L = nt - 1 + 2 * i0, hh = h->h[ax];
        for (int end = 0; end < 2; end++)
            for (int r = 0; r < NR; r++) {
                const int a = end == 0 ? r : nt - NR + r;
                const double ia = a + i0;
                for (int c = 0; c < W; c++) {
                    const int b = a + c - n;
                    if (b < 0 || b >= nt) continue;
                    const double ib = b + i0;
                    const double lo = std::max(0.0, std::max(ia, ib) - s);
                    const double hi = std::min(L, std::min(ia, ib) + s);
                    const double m = half_unit_integral(lo, hi, n, [&](double u) {
                        return bsk::host::bspline(n, u - ia) * bsk::host::bspline(n, u - ib);
                    });
                    const double k = half_unit_integral(lo, hi, n, [&](double u) {
                        return bsk::host::bspline_deriv(n, u - ia) * bsk::host::bspline_deriv(n, u - ib);
                    });
                    const double e = bsk::host::bspline(n, -ia) * bsk::host::bspline(n, -ib) +
                                     bsk::host::bspline(n, L - ia) * bsk::host::bspline(n, L - ib);
                    at(0, ax, end, r, c) = hh * m;
                    at(1, ax, end, r, c) = h->dt * k / hh + h->pen * e;
                }
            }
    }
}

// Per-axis diagonals of the band matrices, [3 axes][2 (mass, dt-weighted stiffness)][jn]: the
// diagonal of the separable operator is their product sum (op_generic.cuh, jacobi_inv). With odd
// reflection a row's own mirror images subtract their taps; Robin rows come from robin_rows.
void jacobi_diagonals(const bsk_handle* h, const std::vector<double>& rows, std::vector<double>& out)
{
    const int n = h->n, NR = n + 1, W = 2 * n + 1;
    out.assign((size_t)6 * h->jn, 1.0);
    for (int ax = 0; ax < 3; ax++) {
        const int nt = dims_of(h, ax);
        for (int pos = 0; pos < nt; pos++) {
            double dm = h->M[ax][n], dk = h->dt * h->K[ax][n];
            if (h->bc == BSK_BC_ROBIN) {
                int end = -1, r = 0;
                if (pos < NR) { end = 0; r = pos; }
                else if (pos >= nt - NR) { end = 1; r = pos - (nt - NR); }
                if (end >= 0) {
                    dm = rows[((((size_t)0 * 3 + ax) * 2 + end) * NR + r) * W + n];
                    dk = rows[((((size_t)1 * 3 + ax) * 2 + end) * NR + r) * W + n];
                }
            } else {
                for (int img : {-2 - pos, 2 * nt - pos}) {
                    const int off = img - pos;
                    if (off >= -n && off <= n) {
                        dm -= h->M[ax][n + off];
                        dk -= h->dt * h->K[ax][n + off];
                    }
                }
            }
            out[((size_t)ax * 2 + 0) * h->jn + pos] = dm;
            out[((size_t)ax * 2 + 1) * h->jn + pos] = dk;
        }
    }
}

// Copies v into dst[0] (float) and dst[1] (double), allocating them on first use.
int upload_both(const std::vector<double>& v, void** dst)
{
    std::vector<float> f(v.begin(), v.end());
    const size_t bytes[2] = {v.size() * sizeof(float), v.size() * sizeof(double)};
    const void* src[2] = {f.data(), v.data()};
    for (int i = 0; i < 2; i++) {
        if (!dst[i]) {
            cudaError_t e = cudaMalloc(&dst[i], bytes[i]);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(BSK_ENOMEM, "table allocation failed");
            }
        }
        BSK_CUDA(cudaMemcpy(dst[i], src[i], bytes[i], cudaMemcpyHostToDevice));
    }
    return BSK_OK;
}

// 1 / diag A per node of the variable-coefficient operator, by probing: the operator is applied
// to the indicator vectors of the (n+1)^3 classes of nodes congruent modulo n + 1 per axis; two
// nodes of one class are more than n apart on some axis (and so are their mirror images), so
// their B-splines do not overlap and each application returns A_ll at every node of its class.
// Runs in the CG precision on the handle's work vectors.
template <typename T>
int probe_diagonal_t(bsk_handle* h)
{
    T* v = static_cast<T*>(h->p0);
    T* y = static_cast<T*>(h->q);
    T* jinv = static_cast<T*>(h->jvec);
    const int s = h->n + 1;
    for (int cz = 0; cz < s; cz++)
        for (int cy = 0; cy < s; cy++)
            for (int cx = 0; cx < s; cx++) {
                BSK_CUDA(bsk::launch_probe<T>(v, y, jinv, 0, h->nx, h->ny, h->nz, s, cx, cy, cz, h->mask, h->stream));
                bsk::OpLaunch L;
                fill_launch(h, L, bsk::MODE_OP);
                L.in0 = v;
                L.out0 = y;
                L.fin = bsk::FIN_NONE;
                BSK_CUDA(bsk::launch_op<T>(L, h->stream));
                BSK_CUDA(bsk::launch_probe<T>(v, y, jinv, 1, h->nx, h->ny, h->nz, s, cx, cy, cz, h->mask, h->stream));
            }
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    return BSK_OK;
}

// 1 / diag A per node of the constant-coefficient operator (Dirichlet or Robin) from the
// per-axis diagonals just uploaded to jac, in the CG precision.
int fill_diagonal(bsk_handle* h)
{
    if (cg_es(h) == sizeof(double))
        BSK_CUDA(bsk::launch_jacobi_fill<double>(static_cast<double*>(h->jvec), h->len, h->nx, h->ny,
                                                 static_cast<const double*>(h->jac[1]), h->jn, h->stream));
    else
        BSK_CUDA(bsk::launch_jacobi_fill<float>(static_cast<float*>(h->jvec), h->len, h->nx, h->ny,
                                                static_cast<const float*>(h->jac[0]), h->jn, h->stream));
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    return BSK_OK;
}

// The per-node inverse diagonal of a Jacobi handle: probed for variable coefficients, formed
// from the separable per-axis diagonals otherwise.
int node_diagonal(bsk_handle* h)
{
    const size_t es = cg_es(h);
    cudaError_t e = cudaMalloc(&h->jvec, h->len * es);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->jvec = nullptr;
        return fail(BSK_ENOMEM, "Jacobi diagonal: cudaMalloc(%zu) failed", h->len * es);
    }
    if (h->cd[0] || h->cd[1]) return es == sizeof(double) ? probe_diagonal_t<double>(h) : probe_diagonal_t<float>(h);
    return fill_diagonal(h);
}

// Rebuilds the Robin rows and Jacobi diagonals after a change of boundary, dt, coefficients or
// preconditioner.
int refresh_tables(bsk_handle* h)
{
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<double> rows;
    if (h->bc == BSK_BC_ROBIN) {
        robin_rows(h, rows);
        if (int rc = upload_both(rows, h->rb)) return rc;
    }
    if (h->pc == BSK_PC_JACOBI) {
        std::vector<double> dg;
        jacobi_diagonals(h, rows, dg);
        if (int rc = upload_both(dg, h->jac)) return rc;
    }
    if (h->jvec) {
        cudaFree(h->jvec);
        h->jvec = nullptr;
    }
    if (h->pc == BSK_PC_JACOBI) return node_diagonal(h);
    return BSK_OK;
}

}  // namespace

extern "C" int bsk_set_dt(bsk_handle* h, double dt)
{
    if (int rc = check_handle(h)) return rc;
    if (!(dt >= 0) || !std::isfinite(dt)) return fail(BSK_EINVAL, "dt must be finite and >= 0");
    if (dt != h->dt && h->graph) {   // the kernels of the captured graph carry dt * K by value
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->dt = dt;
    if (h->bc == BSK_BC_ROBIN || h->pc) return refresh_tables(h);   // their rows carry dt too
    return BSK_OK;
}

extern "C" int bsk_set_boundary(bsk_handle* h, int kind, double penalty)
{
    if (int rc = check_handle(h)) return rc;
    if (kind != BSK_BC_DIRICHLET && kind != BSK_BC_ROBIN) return fail(BSK_EINVAL, "unknown boundary kind %d", kind);
    if (kind == BSK_BC_ROBIN) {
        if (!(penalty >= 0) || !std::isfinite(penalty)) return fail(BSK_EINVAL, "penalty must be finite and >= 0");
        if (h->mask) return fail(BSK_EINVAL, "the Robin boundary is defined on the whole box (no mask)");
        if (h->cd[0] || h->cd[1]) return fail(BSK_EINVAL, "variable coefficients take the Dirichlet boundary");
        if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "the BF16-storage variant has the Dirichlet boundary only");
        for (int ax = 0; ax < 3; ax++)
            if (dims_of(h, ax) < 2 * (h->n + 1))
                return fail(BSK_EINVAL, "a Robin axis needs at least 2 (degree + 1) unknowns");
    }
    h->bc = kind;
    h->pen = kind == BSK_BC_ROBIN ? penalty : 0.0;
    if (kind != BSK_BC_ROBIN)
        for (int i = 0; i < 2; i++)
            if (h->rb[i]) {
                cudaFree(h->rb[i]);
                h->rb[i] = nullptr;
            }
    refresh_paths(h);
    return refresh_tables(h);
}

extern "C" int bsk_set_preconditioner(bsk_handle* h, int kind)
{
    if (int rc = check_handle(h)) return rc;
    if (kind != BSK_PC_NONE && kind != BSK_PC_JACOBI) return fail(BSK_EINVAL, "unknown preconditioner %d", kind);
    if (kind == BSK_PC_JACOBI && h->prec == BSK_BF16S) return fail(BSK_EINVAL, "BF16 storage has no solver");
    h->pc = kind;
    h->jn = std::max(h->nx, std::max(h->ny, h->nz));
    refresh_paths(h);
    return refresh_tables(h);
}

extern "C" int bsk_set_coefficients(bsk_handle* h, const double* d, const double* m)
{
    if (int rc = check_handle(h)) return rc;
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "the BF16-storage variant has constant coefficients only");
    if ((d || m) && h->bc == BSK_BC_ROBIN)
        return fail(BSK_EINVAL, "variable coefficients take the Dirichlet boundary");
    // the captured CG graph holds the kernels of the previous operator
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (!d && !m) {
        for (int i = 0; i < 2; i++) {
            if (h->cd[i]) cudaFree(h->cd[i]);
            if (h->cm[i]) cudaFree(h->cm[i]);
            h->cd[i] = h->cm[i] = nullptr;
        }
        refresh_paths(h);
        return h->pc == BSK_PC_JACOBI ? refresh_tables(h) : BSK_OK;
    }
    const size_t clen = (size_t)(h->nx + 2) * (h->ny + 2) * (h->nz + 2);
    for (int i = 0; i < 2; i++) {
        // FP32 fields for the FP32 passes (BSK_F32, inner solves of BSK_F32_IR), FP64 fields
        // for the FP64 passes (BSK_F64, true residuals of BSK_F32_IR)
        const bool need = i == 0 ? h->prec != BSK_F64 : h->prec != BSK_F32;
        if (!need) continue;
        const size_t bytes = clen * (i == 0 ? sizeof(float) : sizeof(double));
        for (void** f : {&h->cd[i], &h->cm[i]})
            if (!*f) {
                cudaError_t e = cudaMalloc(f, bytes);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(BSK_ENOMEM, "coefficient fields: cudaMalloc(%zu) failed", bytes);
                }
            }
        if (i == 0) {
            BSK_LAUNCH(h, bsk::launch_coef_fill<float>(d, static_cast<float*>(h->cd[0]), clen, h->stream));
            BSK_LAUNCH(h, bsk::launch_coef_fill<float>(m, static_cast<float*>(h->cm[0]), clen, h->stream));
        } else {
            BSK_LAUNCH(h, bsk::launch_coef_fill<double>(d, static_cast<double*>(h->cd[1]), clen, h->stream));
            BSK_LAUNCH(h, bsk::launch_coef_fill<double>(m, static_cast<double*>(h->cm[1]), clen, h->stream));
        }
    }
    // every pass takes the general path, where launch_op dispatches to the variable-coefficient
    // kernel (the right-hand-side mass of heat_step stays the constant mass matrix)
    refresh_paths(h);
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    if (h->pc == BSK_PC_JACOBI) return refresh_tables(h);   // the diagonal changed
    return BSK_OK;
}

extern "C" int bsk_op_flops(bsk_handle* h, double* algorithmic, double* executed)
{
    if (int rc = check_handle(h)) return rc;
    const int n = h->n;
    double alg, exe;
    if (h->cd[0] || h->cd[1]) {
        // per node of an unbounded tile: z-pass 4(n+1) FMA per quad plane, y-pass 5(n+1) FMA + 2
        // products per (qz, qy) node, x-pass 10(n+1) FMA + 4 products per quad point, transposed
        // y- and z-passes 3 Q (n+1) + 2 (n+1) FMA per quad plane
        // (degrees <= 3 fold the quadrature weights: 2 products per y node, 4 per point; else 0, 8)
        const double q = (3 * n + 2) / 2, nb = n + 1;
        const double ny_prod = n <= 3 ? 2 : 0, pt_prod = n <= 3 ? 4 : 8;
        alg = 2.0 * q * 4 * nb + q * q * (2.0 * 5 * nb + ny_prod) + q * q * q * (2.0 * 10 * nb + pt_prod) +
              2.0 * q * (3.0 * q * nb + 2 * nb);
        exe = cg_es(h) == sizeof(double) ? bsk::var_flops_per_node<double>(n, h->nx, h->ny, h->nz)
                                         : bsk::var_flops_per_node<float>(n, h->nx, h->ny, h->nz);
    } else {
        // seven (2n+1)-tap band convolutions per node (the three sweeps of Fig. FiltAlg)
        alg = exe = 14.0 * (2 * n + 1);
    }
    if (algorithmic) *algorithmic = alg;
    if (executed) *executed = exe;
    return BSK_OK;
}

static int apply_common(bsk_handle* h, const void* x, void* y, int mode)
{
    if (int rc = check_handle(h)) return rc;
    if (!x || !y) return fail(BSK_EINVAL, "null vector");
    const size_t es = user_es(h);
    if (overlaps(x, y, h->len * es)) return fail(BSK_EINVAL, "x and y overlap");
    cudaError_t e;
    // op_apply's x is the caller's and may be non-zero off the mask: masked grids take the
    // general kernel, which masks its input
    if (mode == bsk::MODE_OP && !h->mask && tma_ok(h, es, {x, y})) {
        bsk::TmaLaunch T;
        fill_tma(h, T, bsk::TMODE_OP);
        T.in[0] = x;
        T.out0 = y;
        T.fin = bsk::FIN_NONE;
        e = tma_launch_es(es, T, h->stream);
    } else {
        bsk::OpLaunch L;
        fill_launch(h, L, mode);
        L.in0 = x;
        L.out0 = y;
        L.fin = bsk::FIN_NONE;
        if (h->prec == BSK_BF16S) {   // FP32 arithmetic on bfloat16 vectors
            L.bf16io = 1;
            e = bsk::launch_op<float>(L, h->stream);
        } else {
            e = op_launch_es(es, L, h->stream);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "operator launch");
    h->launches += 1;
    return BSK_OK;
}

extern "C" int op_apply(bsk_handle* h, const void* x, void* y)
{
    return apply_common(h, x, y, bsk::MODE_OP);
}

extern "C" int mass_apply(bsk_handle* h, const void* x, void* y)
{
    return apply_common(h, x, y, bsk::MODE_MASS);
}

extern "C" int cg_solve(bsk_handle* h, const void* b, void* x, const bsk_cg_opts* opts,
                        bsk_cg_report* report)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_handle(h)) return rc;
    if (!b || !x) return fail(BSK_EINVAL, "null vector");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "BF16 storage is an operator-only variant");
    if (overlaps(b, x, h->len * user_es(h))) return fail(BSK_EINVAL, "b and x overlap");
    const Opts o = resolve(opts);
    if (report) memset(report, 0, sizeof *report);
    h->launches = 0;
    h->iter_ms = 0.0;
    int st = solve_dispatch(h, b, x, o, report, t0);
    if (report) {
        report->status = st;
        report->elapsed_ms = 1e3 * seconds_since(t0);
        report->kernel_launches = h->launches;
        report->iter_ms = h->iter_ms;
    }
    return st;
}

extern "C" int heat_step(bsk_handle* h, void* u, const void* q, int nsteps, const bsk_cg_opts* opts,
                         bsk_cg_report* report)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_handle(h)) return rc;
    if (!u) return fail(BSK_EINVAL, "null vector");
    if (nsteps < 0) return fail(BSK_EINVAL, "nsteps < 0");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "BF16 storage is an operator-only variant");
    const size_t es = user_es(h);
    if (q && overlaps(u, q, h->len * es)) return fail(BSK_EINVAL, "u and q overlap");
    const Opts o = resolve(opts);
    if (report) memset(report, 0, sizeof *report);
    void* b = h->prec == BSK_F32_IR ? (void*)h->b64 : h->bvec;
    int st = BSK_OK;
    h->launches = 0;
    h->iter_ms = 0.0;
    for (int s = 0; s < nsteps; s++) {
        cudaError_t e;
        if (!q && h->res_df && tma_ok(h, sizeof(double), {u, b})) {
            // M u as the double-float operator with the stiffness weight set to zero; the TMA
            // kernels take inputs that are zero off the mask (the solve below masks u anyway)
            if (h->mask)
                BSK_LAUNCH(h, bsk::launch_copy_masked<double>(static_cast<const double*>(u), static_cast<double*>(u),
                                                         h->len, h->mask, h->stream));
            bsk::TmaLaunch T;
            fill_tma(h, T, bsk::TMODE_OP);
            for (int d = 0; d < 3; d++)
                for (int j = 0; j < bsk::kMaxTaps; j++) T.Kdt[d][j] = 0.0;
            T.in[0] = u;
            T.out0 = b;
            T.fin = bsk::FIN_NONE;
            e = bsk::launch_tma<bsk::dfl>(T, h->stream);
        } else {
            bsk::OpLaunch L;
            fill_launch(h, L, bsk::MODE_MASS);
            L.in0 = u;
            L.in1 = q;
            L.s = h->dt;
            L.out0 = b;
            L.fin = bsk::FIN_NONE;
            e = op_launch_es(es, L, h->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "right-hand side launch");
        h->launches += 1;
        int rs = solve_dispatch(h, b, u, o, report, t0);
        if (rs < 0) { st = rs; break; }
        if (rs > 0 && st == BSK_OK) st = rs;
    }
    if (report) {
        report->status = st;
        report->elapsed_ms = 1e3 * seconds_since(t0);
        report->kernel_launches = h->launches;
        report->iter_ms = h->iter_ms;
    }
    return st;
}

extern "C" int heat_step_host(bsk_handle* h, void* u_host, const void* q_host, int nsteps, const bsk_cg_opts* opts,
                              bsk_cg_report* report)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_handle(h)) return rc;
    if (!u_host) return fail(BSK_EINVAL, "null vector");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "BF16 storage is an operator-only variant");
    const size_t bytes = h->len * user_es(h);
    if (!h->u_dev) {
        BSK_CUDA(cudaMalloc(&h->u_dev, bytes));
        for (int i = 0; i < 4; i++) BSK_CUDA(cudaEventCreate(&h->io_ev[i]));
    }
    if (q_host && !h->q_dev) BSK_CUDA(cudaMalloc(&h->q_dev, bytes));
    BSK_CUDA(cudaEventRecord(h->io_ev[0], h->stream));
    BSK_CUDA(cudaMemcpyAsync(h->u_dev, u_host, bytes, cudaMemcpyHostToDevice, h->stream));
    if (q_host) BSK_CUDA(cudaMemcpyAsync(h->q_dev, q_host, bytes, cudaMemcpyHostToDevice, h->stream));
    BSK_CUDA(cudaEventRecord(h->io_ev[1], h->stream));
    const int st = heat_step(h, h->u_dev, q_host ? h->q_dev : nullptr, nsteps, opts, report);
    if (st < 0) return st;
    BSK_CUDA(cudaEventRecord(h->io_ev[2], h->stream));
    BSK_CUDA(cudaMemcpyAsync(u_host, h->u_dev, bytes, cudaMemcpyDeviceToHost, h->stream));
    BSK_CUDA(cudaEventRecord(h->io_ev[3], h->stream));
    BSK_CUDA(cudaEventSynchronize(h->io_ev[3]));
    if (report) {
        float a = 0.f, b = 0.f;
        BSK_CUDA(cudaEventElapsedTime(&a, h->io_ev[0], h->io_ev[1]));
        BSK_CUDA(cudaEventElapsedTime(&b, h->io_ev[2], h->io_ev[3]));
        report->h2d_ms = a;
        report->d2h_ms = b;
        report->elapsed_ms = 1e3 * seconds_since(t0);
    }
    return st;
}

extern "C" int bsk_net_forward(bsk_net* net, const float* r, const uint8_t* mask, float* z);

// Iterative refinement around the preconditioned inner FCG solve (fcg.cu).
// Flexible CG inside FP64 refinement (fcg_solve); with rec_r set, the first inner solve also
// records its residual and iterate before each of its first rec_steps iterations (fcg_record).
static int fcg_impl(bsk_handle* h, bsk_net* net, const void* bv, void* xv, const Opts& o, bsk_cg_report* rep,
                    std::chrono::steady_clock::time_point t0, float* rec_r, float* rec_x, int rec_steps)
{
    if (rep) memset(rep, 0, sizeof *rep);
    h->launches = 0;
    const double* b = (const double*)bv;
    double* x = (double*)xv;
    if (!h->fcg_ws) {
        cudaError_t e = cudaMalloc((void**)&h->fcg_ws, 3 * h->len * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->fcg_partials, 3 * 1216 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->fcg_state, bsk::fcg_state_bytes());
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BSK_ENOMEM, "FCG work vectors: %s", cudaGetErrorString(e));
        }
        BSK_CUDA(cudaMemsetAsync(h->fcg_state, 0, bsk::fcg_state_bytes(), h->stream));
    }
    bsk::FcgVectors V = {};
    V.b = static_cast<const float*>(h->r);   // the scaled residual is written here, then copied to r
    V.x = static_cast<float*>(h->x);
    V.r = static_cast<float*>(h->r);
    V.p = static_cast<float*>(h->p0);
    V.q = static_cast<float*>(h->q);
    V.z = h->fcg_ws;
    V.rn = h->fcg_ws + h->len;
    V.zn = h->fcg_ws + 2 * h->len;
    V.partials = h->fcg_partials;
    V.state = h->fcg_state;
    V.rec_r = rec_r;
    V.rec_x = rec_x;
    V.rec_steps = rec_steps;
    auto op = [&](const float* p, float* q) -> int {
        cudaError_t e;
        if (tma_ok(h, sizeof(float), {p, q})) {
            bsk::TmaLaunch T;
            fill_tma(h, T, bsk::TMODE_OP);
            T.in[0] = p;
            T.out0 = q;
            T.fin = bsk::FIN_NONE;
            e = bsk::launch_tma<float>(T, h->stream);
        } else {
            bsk::OpLaunch L;
            fill_launch(h, L, bsk::MODE_OP);
            L.in0 = p;
            L.out0 = q;
            L.fin = bsk::FIN_NONE;
            e = bsk::launch_op<float>(L, h->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "operator launch");
        h->launches += 1;
        return BSK_OK;
    };
    auto netf = [&](bsk_net* n, const float* r, const uint8_t* m, float* z) -> int {
        h->launches += 5;
        return bsk_net_forward(n, r, m, z);
    };
    int rc;
    int total_iters = 0, outer = 0, st = BSK_NOT_CONVERGED, fb = -1, total_rejected = 0;
    double rel = 0.0;
    BSK_LAUNCH(h, bsk::launch_copy_masked<double>(x, x, h->len, h->mask, h->stream));
    for (;; outer++) {
        if ((rc = enqueue_residual64(h, b, x, h->r64, h->sc64, o.residual_fp64))) return rc;
        if ((rc = sync_scalars(h, h->sc64))) return rc;
        const double rr = h->h_sc->rr_true, bb = h->h_sc->bb_true;
        if (!std::isfinite(rr) || !std::isfinite(bb)) return fail(BSK_EBREAKDOWN, "non-finite residual");
        if (bb == 0.0) {
            BSK_CUDA(cudaMemsetAsync(x, 0, h->len * sizeof(double), h->stream));
            rel = 0.0;
            st = BSK_OK;
            break;
        }
        rel = std::sqrt(rr / bb);
        if (rel <= o.tol) { st = BSK_OK; break; }
        if (outer >= o.max_outer || total_iters >= o.max_iter) { st = BSK_NOT_CONVERGED; break; }
        double inner = std::max(o.inner_tol, 0.3 * o.tol / rel);
        if (inner > 0.5) inner = 0.5;
        BSK_LAUNCH(h, bsk::launch_ir_scale_down(h->r64, static_cast<float*>(h->r), h->len, h->sc64, h->stream));
        int it = 0, fbi = -1, rej = 0;
        // the network predicts errors in units of 1 / (hx hy hz), the inverse mass scale
        const double out_scale = 1.0 / (h->h[0] * h->h[1] * h->h[2]);
        int ist = bsk::fcg_inner(V, h->len, h->mask, inner, o.max_iter - total_iters, o.stall_window,
                                 out_scale, 0.0, op, net, netf, h->stream, &it, &fbi, &rej, o.time_limit, t0);
        V.rec_r = V.rec_x = nullptr;   // only the first inner solve is recorded
        h->launches += 6LL * it;
        total_iters += it;
        total_rejected += rej;
        if (fbi >= 0) fb = fbi;
        if (ist == BSK_ETIMEOUT || ist == BSK_ECUDA) return ist;
        if (ist == BSK_EBREAKDOWN && it == 0) return ist;
        BSK_LAUNCH(h, bsk::launch_ir_update(x, static_cast<const float*>(h->x), h->len, h->sc64, h->stream));
    }
    if (rep) {
        rep->status = st;
        rep->iterations = total_iters;
        rep->outer_iterations = outer;
        rep->rel_residual = rel;
        rep->elapsed_ms = 1e3 * seconds_since(t0);
        rep->kernel_launches = h->launches;
        rep->fallback_iter = fb;
        rep->net_rejected = total_rejected;
    }
    return st;
}

extern "C" int fcg_solve(bsk_handle* h, bsk_net* net, const void* bv, void* xv, const bsk_cg_opts* opts,
                         bsk_cg_report* rep)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_handle(h)) return rc;
    if (h->prec != BSK_F32_IR) return fail(BSK_EINVAL, "fcg_solve needs a BSK_F32_IR handle");
    if (!bv || !xv) return fail(BSK_EINVAL, "null vector");
    if (overlaps(bv, xv, h->len * sizeof(double))) return fail(BSK_EINVAL, "b and x overlap");
    return fcg_impl(h, net, bv, xv, resolve(opts), rep, t0, nullptr, nullptr, 0);
}

extern "C" int fcg_record(bsk_handle* h, bsk_net* net, const void* bv, int steps, float* r_rec, float* x_rec,
                          double* bnorm, int* recorded)
{
    auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_handle(h)) return rc;
    if (h->prec != BSK_F32_IR) return fail(BSK_EINVAL, "fcg_record needs a BSK_F32_IR handle");
    if (!bv || !r_rec || !x_rec || !bnorm || !recorded || steps < 1) return fail(BSK_EINVAL, "bad argument");
    *recorded = 0;
    // one inner solve of A d = b / ||b|| from d = 0, exactly `steps` iterations unless it breaks
    // down or stalls; x (FP64) lives in the handle's b64 scratch
    Opts o = resolve(nullptr);
    o.tol = 0.0;
    o.inner_tol = 0.0;
    o.max_iter = steps;
    o.max_outer = 1;
    BSK_CUDA(cudaMemsetAsync(h->b64, 0, h->len * sizeof(double), h->stream));
    bsk_cg_report rep;
    const int st = fcg_impl(h, net, bv, h->b64, o, &rep, t0, r_rec, x_rec, steps);
    if (st < 0) return st;
    BSK_CUDA(cudaStreamSynchronize(h->stream));
    *bnorm = std::sqrt(h->h_sc->bb_true);
    *recorded = std::min(rep.iterations + 1, steps);
    return BSK_OK;
}

extern "C" int bsk_inverse_diagonal(bsk_handle* h, void* out)
{
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(BSK_EINVAL, "null vector");
    if (h->prec != BSK_F64 && h->prec != BSK_F32)
        return fail(BSK_EINVAL, "bsk_inverse_diagonal takes BSK_F64 or BSK_F32 handles");
    if (!h->pc || !h->jvec) return fail(BSK_EINVAL, "the handle has no Jacobi preconditioner (bsk_set_preconditioner)");
    if (overlaps(out, h->jvec, h->len * cg_es(h))) return fail(BSK_EINVAL, "out overlaps the handle's diagonal");
    // the handle's vector is not masked (the solvers' residuals are zero off the mask anyway)
    if (cg_es(h) == sizeof(double))
        BSK_CUDA(bsk::launch_copy_masked<double>(static_cast<const double*>(h->jvec), static_cast<double*>(out),
                                                 h->len, h->mask, h->stream));
    else
        BSK_CUDA(bsk::launch_copy_masked<float>(static_cast<const float*>(h->jvec), static_cast<float*>(out),
                                                h->len, h->mask, h->stream));
    return BSK_OK;
}

extern "C" int bsk_time_kernel(bsk_handle* h, int kernel, int reps, double* ms)
{
    if (int rc = check_handle(h)) return rc;
    if (!ms || reps < 1) return fail(BSK_EINVAL, "bad arguments");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "a BF16-storage handle has no solver kernels to time");
    if (kernel < BSK_KERNEL_OP || kernel > BSK_KERNEL_RES_DF) return fail(BSK_EINVAL, "unknown kernel %d", kernel);
    if (kernel == BSK_KERNEL_RES_DF && !h->res_df)
        return fail(BSK_EINVAL, "this handle has no double-float residual kernel");
    if (kernel >= BSK_KERNEL_RES64 && h->prec != BSK_F32_IR)
        return fail(BSK_EINVAL, "the FP64 residual kernel exists only for BSK_F32_IR handles");
    const size_t ces = cg_es(h);
    for (void* p : {h->x, h->r, h->p0, h->p1, h->q, h->r2, h->q2})
        if (p) BSK_CUDA(cudaMemsetAsync(p, 0, h->len * ces, h->stream));
    if (h->r64) BSK_CUDA(cudaMemsetAsync(h->r64, 0, h->len * sizeof(double), h->stream));
    if (h->b64) BSK_CUDA(cudaMemsetAsync(h->b64, 0, h->len * sizeof(double), h->stream));
    if (int rc = init_scalars(h, h->sc_aux, 0.0, 1 << 30, 0)) return rc;
    auto one = [&](int i) -> cudaError_t {
        bsk::OpLaunch L;
        bsk::TmaLaunch T;
        switch (kernel) {
        case BSK_KERNEL_OP:
            if (tma_ok(h, ces, {h->x, h->q})) {
                fill_tma(h, T, bsk::TMODE_OP);
                T.in[0] = h->x;
                T.out0 = h->q;
                T.fin = bsk::FIN_NONE;
                return tma_launch_es(ces, T, h->stream);
            }
            fill_launch(h, L, bsk::MODE_OP);
            L.in0 = h->x;
            L.out0 = h->q;
            L.fin = bsk::FIN_NONE;
            return op_launch_es(ces, L, h->stream);
        case BSK_KERNEL_CG_FUSED:
            if (h->use_tma) {
                fill_tma(h, T, bsk::TMODE_CG);
                cg1_vectors(h, i, T);
                T.sc = h->sc_aux;
                T.partials = h->partials;
                T.fin = bsk::FIN_NORM;   // reduces without touching the CG state of sc
                return tma_launch_es(ces, T, h->stream);
            }
            fill_launch(h, L, bsk::MODE_CGP);
            L.in0 = h->r;
            L.in1 = (i & 1) ? h->p1 : h->p0;
            L.out1 = (i & 1) ? h->p0 : h->p1;
            L.out0 = h->q;
            L.xvec = h->x;
            L.sc = h->sc_aux;
            L.partials = h->partials;
            L.fin = bsk::FIN_NORM;   // reduces p.q without touching the CG state of sc
            return op_launch_es(ces, L, h->stream);
        case BSK_KERNEL_CG_UPDATE:
            return ces == sizeof(double)
                       ? bsk::launch_cg_update<double>((double*)h->r, (const double*)h->q, h->len,
                                                       h->sc_aux, h->partials, bsk::FIN_NORM, h->stream)
                       : bsk::launch_cg_update<float>((float*)h->r, (const float*)h->q, h->len,
                                                      h->sc_aux, h->partials, bsk::FIN_NORM, h->stream);
        default:  // BSK_KERNEL_RES64, BSK_KERNEL_RES_DF
            if (tma_ok(h, sizeof(double), {h->b64, h->r64})) {
                fill_tma(h, T, bsk::TMODE_RES);
                T.in[0] = h->b64;
                T.inint = h->b64;
                T.out0 = h->r64;
                T.sc = h->sc_aux;
                T.partials = h->partials;
                T.fin = bsk::FIN_RES_TRUE;
                return kernel == BSK_KERNEL_RES_DF ? bsk::launch_tma<bsk::dfl>(T, h->stream)
                                                   : bsk::launch_tma<double>(T, h->stream);
            }
            fill_launch(h, L, bsk::MODE_RES);
            L.in0 = h->b64;
            L.b = h->b64;
            L.out0 = h->r64;
            L.sc = h->sc_aux;
            L.partials = h->partials;
            L.fin = bsk::FIN_RES_TRUE;
            return op_launch_es(sizeof(double), L, h->stream);
        }
    };
    // one untimed launch (first-launch set-up), then the timed batch
    BSK_CUDA(one(0));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BSK_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < reps && err == cudaSuccess; i++) err = one(i + 1);
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float total = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&total, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "bsk_time_kernel");
    *ms = (double)total / reps;
    return BSK_OK;
}

extern "C" int bsk_cg_kernel_config(bsk_handle* h, int* kernel, int* zchunk_planes)
{
    if (int rc = check_handle(h)) return rc;
    if (kernel) *kernel = h->cg_impl == 0 ? BSK_CG_KERNEL_WS : BSK_CG_KERNEL_CLASSIC;
    if (zchunk_planes) *zchunk_planes = h->cg_impl == 0 ? (h->ws_chunk > 0 ? h->ws_chunk : 128) : 0;
    return BSK_OK;
}

extern "C" int bsk_select_cg_kernel(bsk_handle* h, int request, int* chosen)
{
    if (int rc = check_handle(h)) return rc;
    if (request != BSK_CG_KERNEL_AUTO && request != BSK_CG_KERNEL_WS && request != BSK_CG_KERNEL_CLASSIC &&
        request != BSK_CG_KERNEL_CURRENT && request != BSK_CG_KERNEL_WS_CHUNKED &&
        request != BSK_CG_KERNEL_WS_COLUMNS)
        return fail(BSK_EINVAL, "unknown CG kernel request %d", request);
    if (request == BSK_CG_KERNEL_CURRENT) {
        if (chosen) *chosen = h->cg_impl == 0 ? BSK_CG_KERNEL_WS : BSK_CG_KERNEL_CLASSIC;
        return BSK_OK;
    }
    const bool ws_ok = cg_ws_eligible(h);
    const bool ws_req = request == BSK_CG_KERNEL_WS || request == BSK_CG_KERNEL_WS_CHUNKED ||
                        request == BSK_CG_KERNEL_WS_COLUMNS;
    if (ws_req && !ws_ok)
        return fail(BSK_EINVAL, "the warp-specialised CG pass needs an unmasked FP32 TMA grid of degree <= 4");
    int impl = ws_req ? 0 : 1, chunk = request == BSK_CG_KERNEL_WS_COLUMNS ? h->nz : 0;
    if ((request == BSK_CG_KERNEL_AUTO || request == BSK_CG_KERNEL_WS) && ws_ok) {
        // time the candidates on the handle's own vectors (bsk_time_kernel zeroes them first and
        // launches once untimed); the first measurement of each warms it up. The warp-specialised
        // pass runs with z-chunks of at most 128 planes and with whole columns (the chunk cap
        // at nz): which is faster depends on how many rounds of items the grid makes.
        struct Cand { int impl, chunk; };
        const Cand cands[3] = {{0, 0}, {0, h->nz}, {1, 0}};
        const int ncand = request == BSK_CG_KERNEL_AUTO ? 3 : 2;
        const bool tma_now = h->use_tma;
        h->use_tma = h->use_tma0;
        double best = 0.0;
        for (int c = 0; c < ncand; c++) {
            h->cg_impl = cands[c].impl;
            h->ws_chunk = cands[c].chunk;
            double ms = 0.0;
            int rc = bsk_time_kernel(h, BSK_KERNEL_CG_FUSED, 1, &ms);
            if (rc == BSK_OK) rc = bsk_time_kernel(h, BSK_KERNEL_CG_FUSED, 2, &ms);
            if (rc != BSK_OK) {
                h->use_tma = tma_now;
                return rc;
            }
            if (c == 0 || ms < best) {
                best = ms;
                impl = cands[c].impl;
                chunk = cands[c].chunk;
            }
        }
        h->use_tma = tma_now;
    }
    h->cg_impl = impl;
    h->ws_chunk = chunk;
    if (h->graph) {   // the captured CG chunk holds the previous kernel
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (chosen) *chosen = impl == 0 ? BSK_CG_KERNEL_WS : BSK_CG_KERNEL_CLASSIC;
    return BSK_OK;
}

// ---- B-spline transforms at the nodes -------------------------------------------------------

namespace {

int transform_halfwidth(int n) { return (n + 2) / 2 - 1; }   // ceil((n + 1) / 2) - 1

// Banded Cholesky factor of the sampled odd-reflected basis of one axis with N unknowns:
// B[j][i] = sum over the images of unknown i (i + 1 + m P with sign +, -(i + 1) + m P with sign
// -, P = 2 (N + 1), m = -1, 0, 1) of beta^n(j + 1 - image). Row j of the output holds
// { 1 / L[j][j], L[j][j-1], ..., L[j][j-p] }. Returns false if B is not positive definite.
bool sampled_basis_cholesky(int n, int N, std::vector<double>& out)
{
    const int p = transform_halfwidth(n), w = p + 1;
    const long long P = 2LL * (N + 1);
    auto b = [&](int j, int i) {
        const long long J = j + 1, I = i + 1;
        const long long img[6] = {I, I + P, I - P, -I, -I + P, -I - P};
        double v = 0.0;
        for (int q = 0; q < 6; q++) {
            const long long d = J - img[q];
            if (d >= -p && d <= p) v += (q < 3 ? 1.0 : -1.0) * bspline_at(n, (int)d);
        }
        return v;
    };
    std::vector<double> Lf((size_t)N * w, 0.0);   // Lf[j * w + (j - k)] = L[j][k]
    auto Lat = [&](int j, int k) -> double& { return Lf[(size_t)j * w + (j - k)]; };
    for (int j = 0; j < N; j++) {
        for (int k = std::max(0, j - p); k <= j; k++) {
            double sum = b(j, k);
            for (int m = std::max(0, j - p); m < k; m++)
                if (m >= k - p) sum -= Lat(j, m) * Lat(k, m);
            if (k == j) {
                if (!(sum > 0.0)) return false;
                Lat(j, j) = std::sqrt(sum);
            } else {
                Lat(j, k) = sum / Lat(k, k);
            }
        }
    }
    out.assign((size_t)N * w, 0.0);
    for (int j = 0; j < N; j++) {
        out[(size_t)j * w] = 1.0 / Lat(j, j);
        for (int k = 1; k <= p && j - k >= 0; k++) out[(size_t)j * w + k] = Lat(j, j - k);
    }
    return true;
}

}  // namespace

extern "C" int bsk_transform(bsk_handle* h, int direction, const void* in, void* out)
{
    if (int rc = check_handle(h)) return rc;
    if (h->bc == BSK_BC_ROBIN) return fail(BSK_EINVAL, "the transforms take the Dirichlet (reflected) basis");
    if (!in || !out) return fail(BSK_EINVAL, "null vector");
    if (direction != BSK_TO_SAMPLES && direction != BSK_TO_COEFFS)
        return fail(BSK_EINVAL, "unknown transform direction %d", direction);
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "the transforms take FP32 or FP64 vectors");
    const size_t es = user_es(h);
    if (overlaps(in, out, h->len * es)) return fail(BSK_EINVAL, "in and out overlap");
    const int n = h->n, p = transform_halfwidth(n);
    if (direction == BSK_TO_SAMPLES) {
        // u = (Bz (x) By (x) Bx) c: the mass-only sweeps with the sampled B-spline as taps
        bsk::OpLaunch L;
        fill_launch(h, L, bsk::MODE_MASS);
        L.mask = nullptr;   // the transform acts on the whole box
        for (int d = 0; d < 3; d++)
            for (int j = 0; j < bsk::kMaxTaps; j++) {
                const int off = j - n;
                L.M[d][j] = (off >= -p && off <= p) ? bspline_at(n, off) : 0.0;
                L.Kdt[d][j] = 0.0;
            }
        L.in0 = in;
        L.in1 = nullptr;
        L.s = 0.0;
        L.out0 = out;
        L.fin = bsk::FIN_NONE;
        BSK_LAUNCH(h, op_launch_es(es, L, h->stream));
        return BSK_OK;
    }
    // c = (Bz^-1 (x) By^-1 (x) Bx^-1) f: copy, then banded solves along x, y and z
    const int dims[3] = {h->nx, h->ny, h->nz};
    if (p > 0 && !h->tr_L[0]) {
        for (int d = 0; d < 3; d++) {
            std::vector<double> f;
            if (!sampled_basis_cholesky(n, dims[d], f)) return fail(BSK_EBREAKDOWN, "sampled basis not positive definite");
            void* dev = nullptr;
            const size_t bytes = f.size() * es;
            BSK_CUDA(cudaMalloc(&dev, bytes));
            h->tr_L[d] = dev;
            if (es == sizeof(double)) {
                BSK_CUDA(cudaMemcpy(dev, f.data(), bytes, cudaMemcpyHostToDevice));
            } else {
                std::vector<float> ff(f.begin(), f.end());
                BSK_CUDA(cudaMemcpy(dev, ff.data(), bytes, cudaMemcpyHostToDevice));
            }
        }
    }
    BSK_CUDA(cudaMemcpyAsync(out, in, h->len * es, cudaMemcpyDeviceToDevice, h->stream));
    if (p > 0)
        for (int d = 0; d < 3; d++) {
            if (es == sizeof(double))
                BSK_LAUNCH(h, bsk::launch_band_solve<double>(static_cast<double*>(out), h->nx, h->ny, h->nz, d, p,
                                                            static_cast<const double*>(h->tr_L[d]), h->stream));
            else
                BSK_LAUNCH(h, bsk::launch_band_solve<float>(static_cast<float*>(out), h->nx, h->ny, h->nz, d, p,
                                                           static_cast<const float*>(h->tr_L[d]), h->stream));
        }
    return BSK_OK;
}

// ---- coarse-to-fine prolongation of Robin problems --------------------------------------------

namespace {

// 1-D transfer between the Robin bases of a fine and a coarse grid on the same interval [0, L]:
// T[f][c] = int_0^L beta(x/hf - if) beta(x/hc - ic) dx for the coarse columns c0[f] .. c0[f]+w-1
// whose supports meet that of fine function f. Between consecutive breakpoints of either grid (the
// half-multiples of hf and of hc) the integrand is one polynomial of degree 2n, integrated exactly
// by n + 1 Gauss points.
void transfer_1d(int n, int ntf, double hf, int ntc, double hc, std::vector<double>& tab, std::vector<int>& c0,
                 int& w)
{
    const int i0 = -(n / 2);
    const double s = 0.5 * (n + 1), L = (ntf - 1 + 2 * i0) * hf;
    std::vector<int> lo(ntf, 0), hi(ntf, 0);
    w = 1;
    for (int f = 0; f < ntf; f++) {
        const double xf = (f + i0) * hf;
        int cl = ntc, ch = -1;
        for (int c = 0; c < ntc; c++)
            if (std::fabs(xf - (c + i0) * hc) < s * (hf + hc)) {
                cl = std::min(cl, c);
                ch = std::max(ch, c);
            }
        if (ch < cl) cl = ch = 0;
        lo[f] = cl;
        hi[f] = ch;
        w = std::max(w, ch - cl + 1);
    }
    tab.assign((size_t)ntf * w, 0.0);
    c0 = lo;
    double xi[16], wt[16];
    bsk::host::gauss_unit(n + 1, xi, wt);
    std::vector<double> br;
    for (int f = 0; f < ntf; f++) {
        const double xf = (f + i0) * hf;
        for (int c = lo[f]; c <= hi[f]; c++) {
            const double xc = (c + i0) * hc;
            const double a = std::max(0.0, std::max(xf - s * hf, xc - s * hc));
            const double b = std::min(L, std::min(xf + s * hf, xc + s * hc));
            if (!(b > a)) continue;
            br.assign({a, b});
            for (double step : {0.5 * hf, 0.5 * hc})
                for (long long k = (long long)std::ceil(a / step); k * step < b; k++)
                    if (k * step > a) br.push_back(k * step);
            std::sort(br.begin(), br.end());
            double acc = 0.0;
            for (size_t j = 0; j + 1 < br.size(); j++) {
                const double p0 = br[j], len = br[j + 1] - br[j];
                if (!(len > 1e-15 * L)) continue;
                for (int g = 0; g <= n; g++) {
                    const double x = p0 + len * xi[g];
                    acc += len * wt[g] * bsk::host::bspline(n, x / hf - (f + i0)) * bsk::host::bspline(n, x / hc - (c + i0));
                }
            }
            tab[(size_t)f * w + (c - lo[f])] = acc;
        }
    }
}

// Banded Cholesky factor of the 1-D Robin Gram matrix of one axis (half-width n): interior rows the
// shift-invariant mass kernel, the N + 1 rows at each end from robin_rows. Row j of the output is
// { 1 / L[j][j], L[j][j-1], ..., L[j][j-n] }. False if not positive definite.
bool robin_gram_cholesky(const bsk_handle* h, int ax, const std::vector<double>& rows, std::vector<double>& out)
{
    const int n = h->n, nt = dims_of(h, ax), NR = n + 1, W = 2 * n + 1, w = n + 1;
    auto Mab = [&](int a, int b) -> double {   // |a - b| <= n
        const int c = b - a + n;
        if (a < NR) return rows[((((size_t)0 * 3 + ax) * 2 + 0) * NR + a) * W + c];
        if (a >= nt - NR) return rows[((((size_t)0 * 3 + ax) * 2 + 1) * NR + (a - (nt - NR))) * W + c];
        return h->M[ax][c];
    };
    std::vector<double> Lf((size_t)nt * w, 0.0);
    auto Lat = [&](int j, int k) -> double& { return Lf[(size_t)j * w + (j - k)]; };
    for (int j = 0; j < nt; j++)
        for (int k = std::max(0, j - n); k <= j; k++) {
            double sum = Mab(j, k);
            for (int m = std::max(0, j - n); m < k; m++)
                if (m >= k - n) sum -= Lat(j, m) * Lat(k, m);
            if (k == j) {
                if (!(sum > 0.0)) return false;
                Lat(j, j) = std::sqrt(sum);
            } else {
                Lat(j, k) = sum / Lat(k, k);
            }
        }
    out.assign((size_t)nt * w, 0.0);
    for (int j = 0; j < nt; j++) {
        out[(size_t)j * w] = 1.0 / Lat(j, j);
        for (int k = 1; k <= n && j - k >= 0; k++) out[(size_t)j * w + k] = Lat(j, j - k);
    }
    return true;
}

template <typename T>
int prolong_impl(bsk_handle* fh, bsk_handle* ch, const T* xc, T* xf)
{
    const int n = fh->n;
    std::vector<double> rows;
    robin_rows(fh, rows);
    int nf[3], nc[3], w[3];
    std::vector<void*> dev;
    auto cleanup = [&]() {
        cudaStreamSynchronize(fh->stream);
        for (void* p : dev) cudaFree(p);
    };
    auto put = [&](const void* src, size_t bytes) -> void* {
        void* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        dev.push_back(d);
        if (src && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return d;
    };
    T* tab[3];
    int* c0d[3];
    T* Ld[3];
    for (int ax = 0; ax < 3; ax++) {
        nf[ax] = dims_of(fh, ax);
        nc[ax] = dims_of(ch, ax);
        std::vector<double> t, lr;
        std::vector<int> c0;
        transfer_1d(n, nf[ax], fh->h[ax], nc[ax], ch->h[ax], t, c0, w[ax]);
        if (!robin_gram_cholesky(fh, ax, rows, lr)) {
            cleanup();
            return fail(BSK_EINVAL, "the fine Gram matrix is not positive definite");
        }
        std::vector<T> tt(t.begin(), t.end()), ll(lr.begin(), lr.end());
        tab[ax] = static_cast<T*>(put(tt.data(), tt.size() * sizeof(T)));
        c0d[ax] = static_cast<int*>(put(c0.data(), c0.size() * sizeof(int)));
        Ld[ax] = static_cast<T*>(put(ll.data(), ll.size() * sizeof(T)));
        if (!tab[ax] || !c0d[ax] || !Ld[ax]) {
            cleanup();
            return fail(BSK_ENOMEM, "prolongation tables");
        }
    }
    T* t1 = static_cast<T*>(put(nullptr, (size_t)nf[0] * nc[1] * nc[2] * sizeof(T)));
    T* t2 = static_cast<T*>(put(nullptr, (size_t)nf[0] * nf[1] * nc[2] * sizeof(T)));
    if (!t1 || !t2) {
        cleanup();
        return fail(BSK_ENOMEM, "prolongation work arrays");
    }
    cudaStream_t s = fh->stream;
    cudaError_t e = bsk::launch_transfer<T>(xc, t1, nc[0], nc[1], nc[2], 0, nf[0], w[0], tab[0], c0d[0], s);
    if (e == cudaSuccess) e = bsk::launch_transfer<T>(t1, t2, nf[0], nc[1], nc[2], 1, nf[1], w[1], tab[1], c0d[1], s);
    if (e == cudaSuccess) e = bsk::launch_transfer<T>(t2, xf, nf[0], nf[1], nc[2], 2, nf[2], w[2], tab[2], c0d[2], s);
    for (int ax = 0; ax < 3 && e == cudaSuccess; ax++)
        e = bsk::launch_band_solve<T>(xf, nf[0], nf[1], nf[2], ax, n, Ld[ax], s);
    fh->launches += 6;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "prolongation");
    return BSK_OK;
}

}  // namespace

extern "C" int bsk_prolong(bsk_handle* fine, bsk_handle* coarse, const void* xc, void* xf)
{
    if (int rc = check_handle(fine)) return rc;
    if (int rc = check_handle(coarse)) return rc;
    if (!xc || !xf) return fail(BSK_EINVAL, "null vector");
    if (fine->bc != BSK_BC_ROBIN || coarse->bc != BSK_BC_ROBIN)
        return fail(BSK_EINVAL, "bsk_prolong takes two Robin handles");
    if (fine->n != coarse->n) return fail(BSK_EINVAL, "the two handles have different degrees");
    if (user_es(fine) != user_es(coarse)) return fail(BSK_EINVAL, "the two handles have different element types");
    const int i0 = -(fine->n / 2);
    for (int ax = 0; ax < 3; ax++) {
        const double lf = (dims_of(fine, ax) - 1 + 2 * i0) * fine->h[ax];
        const double lc = (dims_of(coarse, ax) - 1 + 2 * i0) * coarse->h[ax];
        if (!(std::fabs(lf - lc) <= 1e-12 * lf)) return fail(BSK_EINVAL, "the two grids cover different boxes");
    }
    // the coarse handle's stream must be done with xc before the fine stream reads it
    BSK_CUDA(cudaStreamSynchronize(coarse->stream));
    fine->launches = 0;
    if (user_es(fine) == sizeof(double))
        return prolong_impl<double>(fine, coarse, static_cast<const double*>(xc), static_cast<double*>(xf));
    // FP32 handles: the transfers and line solves run in FP64 (the Gram matrices of the
    // untruncated basis are ill-conditioned for n >= 2: FP32 line solves lost 3 % at n = 3) and
    // the result is rounded once
    double *c64 = nullptr, *f64 = nullptr;
    cudaError_t e = cudaMalloc((void**)&c64, coarse->len * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&f64, fine->len * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c64) cudaFree(c64);
        return fail(BSK_ENOMEM, "prolongation work arrays");
    }
    int rc = BSK_OK;
    e = bsk::launch_convert_f32_f64(static_cast<const float*>(xc), c64, coarse->len, fine->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "prolongation");
    if (rc == BSK_OK) rc = prolong_impl<double>(fine, coarse, c64, f64);
    if (rc == BSK_OK) {
        e = bsk::launch_convert_f64_f32(f64, static_cast<float*>(xf), fine->len, fine->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(fine->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "prolongation");
    }
    cudaStreamSynchronize(fine->stream);
    cudaFree(c64);
    cudaFree(f64);
    return rc;
}

extern "C" int bsk_residual(bsk_handle* h, const void* b, const void* x, void* r, int fp64, double* rr,
                            double* bb)
{
    if (int rc = check_handle(h)) return rc;
    if (!b || !x || !r) return fail(BSK_EINVAL, "null vector");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "BF16 storage is an operator-only variant");
    const size_t es = user_es(h);
    if (overlaps(r, x, h->len * es) || overlaps(r, b, h->len * es)) return fail(BSK_EINVAL, "r overlaps b or x");
    h->launches = 0;
    int rc;
    // the TMA kernels leave the items without active nodes unwritten: the caller's r is
    // zeroed first so that it reads zero off the mask
    if (h->occ) BSK_CUDA(cudaMemsetAsync(r, 0, h->len * es, h->stream));
    if (es == sizeof(double)) {
        if ((rc = enqueue_residual64(h, (const double*)b, (const double*)x, (double*)r, h->sc_aux, fp64 != 0)))
            return rc;
    } else if (tma_ok(h, sizeof(float), {b, x, r})) {
        bsk::TmaLaunch R;
        fill_tma(h, R, bsk::TMODE_RES);
        R.in[0] = x;
        R.inint = b;
        R.out0 = r;
        R.sc = h->sc_aux;
        R.partials = h->partials;
        R.fin = bsk::FIN_RES_TRUE;
        BSK_LAUNCH(h, bsk::launch_tma<float>(R, h->stream));
    } else {
        bsk::OpLaunch L;
        fill_launch(h, L, bsk::MODE_RES);
        L.in0 = x;
        L.b = b;
        L.out0 = r;
        L.sc = h->sc_aux;
        L.partials = h->partials;
        L.fin = bsk::FIN_RES_TRUE;
        BSK_LAUNCH(h, op_launch<float>(L, h->stream));
    }
    if ((rc = sync_scalars(h, h->sc_aux))) return rc;
    if (rr) *rr = h->h_sc->rr_true;
    if (bb) *bb = h->h_sc->bb_true;
    return BSK_OK;
}

extern "C" int bsk_norm2(bsk_handle* h, const void* x, double* out)
{
    if (int rc = check_handle(h)) return rc;
    if (!x || !out) return fail(BSK_EINVAL, "null argument");
    if (h->prec == BSK_BF16S) return fail(BSK_EINVAL, "bsk_norm2 takes FP32 or FP64 vectors");
    cudaError_t e = user_es(h) == sizeof(double)
                        ? bsk::launch_norm2<double>((const double*)x, h->len, h->sc_aux, h->partials, h->stream)
                        : bsk::launch_norm2<float>((const float*)x, h->len, h->sc_aux, h->partials, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "norm launch");
    if (int rc = sync_scalars(h, h->sc_aux)) return rc;
    *out = h->h_sc->rr_true;
    return BSK_OK;
}

// ---- z-slab split (section 3: one problem distributed over several GPUs, here by z-planes) ----

namespace {

int check_slab(const bsk_handle* h)
{
    if (int rc = check_handle(h)) return rc;
    if (h->nz_glob <= 0) return fail(BSK_EINVAL, "the handle has no slab placement (bsk_set_slab)");
    return BSK_OK;
}

size_t plane_len(const bsk_handle* h) { return (size_t)h->nx * h->ny; }

// Local planes of a halo-extended slab vector (n halo planes first).
const void* slab_local(const bsk_handle* h, const void* v_halo)
{
    return static_cast<const char*>(v_halo) + (size_t)h->n * plane_len(h) * user_es(h);
}

int slab_pass_es(bsk_handle* h, int pass, const bsk::SlabVectors& v, double* s)
{
    if (!s) return fail(BSK_EINVAL, "null scalar array");
    const cudaError_t e = user_es(h) == sizeof(double)
                              ? bsk::slab_pass<double>(pass, v, h->len, s, h->slab_partials, h->slab_ctr, h->stream)
                              : bsk::slab_pass<float>(pass, v, h->len, s, h->slab_partials, h->slab_ctr, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab CG pass");
    h->launches += 1;
    return BSK_OK;
}

}  // namespace

extern "C" int bsk_set_slab(bsk_handle* h, int z_off, int nz_glob)
{
    if (int rc = check_handle(h)) return rc;
    if (h->prec != BSK_F64 && h->prec != BSK_F32)
        return fail(BSK_EINVAL, "slab handles take precision BSK_F64 or BSK_F32");
    if (h->mask || h->bc != BSK_BC_DIRICHLET || h->cd[0] || h->cd[1])
        return fail(BSK_EINVAL, "slab handles take unmasked, constant-coefficient grids with odd reflection");
    if (z_off < 0 || nz_glob < 1 || (long long)z_off + h->nz > nz_glob)
        return fail(BSK_EINVAL, "slab planes %d..%d do not lie in a grid of %d planes", z_off, z_off + h->nz - 1,
                    nz_glob);
    if (!h->slab_partials) {
        BSK_CUDA(cudaMalloc((void**)&h->slab_partials, bsk::slab_partials_doubles() * sizeof(double)));
        BSK_CUDA(cudaMalloc((void**)&h->slab_ctr, sizeof(unsigned)));
        BSK_CUDA(cudaMemsetAsync(h->slab_ctr, 0, sizeof(unsigned), h->stream));
    }
    h->z_off = z_off;
    h->nz_glob = nz_glob;
    return BSK_OK;
}

extern "C" int bsk_slab_apply(bsk_handle* h, const void* x_halo, void* y)
{
    if (int rc = check_slab(h)) return rc;
    if (!x_halo || !y) return fail(BSK_EINVAL, "null vector");
    const size_t es = user_es(h);
    const size_t in_bytes = (size_t)(h->nz + 2 * h->n) * plane_len(h) * es;
    const char *a = (const char*)x_halo, *b = (const char*)y;
    if (a < b + h->len * es && b < a + in_bytes) return fail(BSK_EINVAL, "x_halo and y overlap");
    cudaError_t e;
    if (tma_ok(h, es, {x_halo, y})) {   // 16-byte rows: the TMA operator kernel
        bsk::TmaLaunch T;
        fill_tma(h, T, bsk::TMODE_OP);
        T.in[0] = x_halo;
        T.out0 = y;
        T.fin = bsk::FIN_NONE;
        T.z_off = h->z_off;
        T.nz_glob = h->nz_glob;
        T.zpad = h->n;
        e = tma_launch_es(es, T, h->stream);
    } else {
        bsk::OpLaunch L;
        fill_launch(h, L, bsk::MODE_OP);
        L.in0 = x_halo;
        L.out0 = y;
        L.fin = bsk::FIN_NONE;
        L.z_off = h->z_off;
        L.nz_glob = h->nz_glob;
        L.zpad = h->n;
        e = op_launch_es(es, L, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "slab operator launch");
    h->launches += 1;
    return BSK_OK;
}

extern "C" int bsk_slab_cg_begin(bsk_handle* h, const void* b, const void* ax, void* r, void* p_halo, double* s,
                                 double tol, int max_iter)
{
    if (int rc = check_slab(h)) return rc;
    if (!b || !ax || !r || !p_halo || !s) return fail(BSK_EINVAL, "null argument");
    if (!(tol >= 0.0) || max_iter < 0) return fail(BSK_EINVAL, "tol must be >= 0 and max_iter >= 0");
    double init[BSK_SLAB_SCALARS] = {};
    init[BSK_SLAB_TOL2] = tol * tol;
    init[BSK_SLAB_MAX_ITER] = (double)max_iter;
    // pageable source: the copy has left `init` when cudaMemcpyAsync returns
    BSK_CUDA(cudaMemcpyAsync(s, init, sizeof init, cudaMemcpyHostToDevice, h->stream));
    bsk::SlabVectors v = {};
    v.b = b;
    v.ax = ax;
    v.r = r;
    v.p = const_cast<void*>(slab_local(h, p_halo));
    return slab_pass_es(h, bsk::SLAB_BEGIN, v, s);
}

extern "C" int bsk_slab_cg_matvec(bsk_handle* h, const void* p_halo, void* q, double* s)
{
    if (int rc = bsk_slab_apply(h, p_halo, q)) return rc;
    bsk::SlabVectors v = {};
    v.p = const_cast<void*>(slab_local(h, p_halo));
    v.q = q;
    return slab_pass_es(h, bsk::SLAB_DOT, v, s);
}

extern "C" int bsk_slab_cg_update(bsk_handle* h, void* x, void* r, const void* p_halo, const void* q, double* s)
{
    if (int rc = check_slab(h)) return rc;
    if (!x || !r || !p_halo || !q) return fail(BSK_EINVAL, "null vector");
    bsk::SlabVectors v = {};
    v.x = x;
    v.r = r;
    v.p = const_cast<void*>(slab_local(h, p_halo));
    v.q = q;
    return slab_pass_es(h, bsk::SLAB_UPDATE, v, s);
}

extern "C" int bsk_slab_cg_direction(bsk_handle* h, const void* r, void* p_halo, double* s, int first)
{
    if (int rc = check_slab(h)) return rc;
    if (!r || !p_halo) return fail(BSK_EINVAL, "null vector");
    bsk::SlabVectors v = {};
    v.r = const_cast<void*>(r);
    v.p = const_cast<void*>(slab_local(h, p_halo));
    return slab_pass_es(h, first ? bsk::SLAB_FIRST : bsk::SLAB_DIRECTION, v, s);
}

extern "C" const char* bsk_last_error(void) { return g_err.c_str(); }

extern "C" const char* bsk_status_string(int s)
{
    switch (s) {
    case BSK_OK: return "ok";
    case BSK_NOT_CONVERGED: return "not converged (max_iter)";
    case BSK_STALLED: return "stalled";
    case BSK_EINVAL: return "invalid argument";
    case BSK_ECUDA: return "CUDA error";
    case BSK_ENOMEM: return "out of memory";
    case BSK_ETIMEOUT: return "time limit exceeded";
    case BSK_EBREAKDOWN: return "breakdown";
    default: return "unknown status";
    }
}

// ---- helpers shared with the other translation units ----------------------------------------
namespace bsk {

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

dim3 op_grid(int nx, int ny, int nz, int degree, int* tz)
{
    (void)degree;
    const int bx = (nx + kGenTX - 1) / kGenTX, by = (ny + kGenTY - 1) / kGenTY;
    const long long bxy = (long long)bx * by;
    // enough blocks for several waves on 152 SMs, but at least 16 planes per block so that the
    // 2n halo planes re-staged per block stay a small overhead
    long long nzc = (1216 + bxy - 1) / bxy;
    int t = (int)((nz + nzc - 1) / nzc);
    if (t < 16) t = 16;
    if (t > nz) t = nz;
    *tz = t;
    return dim3(bx, by, (nz + t - 1) / t);
}

size_t op_grid_blocks(int nx, int ny, int nz, int degree)
{
    int tz;
    dim3 g = op_grid(nx, ny, nz, degree, &tz);
    return (size_t)g.x * g.y * g.z;
}

int vec_grid(size_t len)
{
    size_t b = (len + 4 * 256 - 1) / (4 * 256);
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace bsk
