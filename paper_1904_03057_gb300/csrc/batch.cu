// batch.cu -- many independent heat problems solved together (bsk_batch_* in include/bsk.h).
//
// Every problem keeps its FP32 CG vectors in a row-padded layout (rows rounded up to 16-byte
// multiples, so any nx is TMA-addressable). One CG iteration of the whole batch is one
// persistent launch per B-spline degree present: the blocks of that launch take (problem, tile,
// z-chunk) items from a device queue, run the single-pass iteration of op_tma.cuh on them, and
// the block finishing a problem's last item reduces that problem's dot products and updates its
// scalars; converged problems drop out of the queue. A CUDA graph holds `check_every`
// iterations; the host polls one status array per graph launch. Around the FP32 iteration the
// FP64 true residual and update of iterative refinement run per problem, in lockstep. An
// autotuner times, per degree, the tile shape (64 x 16, 24 or 32) and z-chunks per problem, and
// derives the graph length.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bsk.h"
#include "bsk_launch.h"

using bsk::Scalars;

namespace {

// r32 (row-padded) = r64 (dense) / ||r64||; the padding is written as zero.
__global__ void k_pack_scaled(const double* __restrict__ r64, float* __restrict__ r32, int nx, int ny,
                              int nz, int pitch, const Scalars* outer)
{
    const double inv = 1.0 / sqrt(outer->rr_true);
    const size_t total = (size_t)nz * ny * pitch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % pitch);
        const size_t row = i / pitch;
        r32[i] = c < nx ? (float)(r64[row * nx + c] * inv) : 0.f;
    }
}

// x64 (dense) += ||r64|| d32 (row-padded).
__global__ void k_unpack_update(double* __restrict__ x64, const float* __restrict__ d32, int nx, int ny,
                                int nz, int pitch, const Scalars* outer)
{
    const double s = sqrt(outer->rr_true);
    const size_t total = (size_t)nz * ny * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const int c = (int)(i - row * nx);
        x64[i] = fma(s, (double)d32[row * pitch + c], x64[i]);
    }
}

int grid_for(size_t n)
{
    size_t b = (n + 1023) / 1024;
    return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 8));
}

struct Prob {
    int nx, ny, nz, n, pitch;
    double h[3];
    double M[3][bsk::kMaxTaps], K[3][bsk::kMaxTaps];
    size_t len, plen;              // dense / padded element counts
    float *r[2], *q[2], *p[2], *x;
    double *r64, *b64;
    double* partials64;            // general-kernel residual reductions
    int nzc;                       // z-chunks per problem (autotuned)
};

struct Group {
    int degree = 0;
    int rows = 3;                  // output rows per warp of the group's tiles (tile 64 x 8 rows)
    int nzc = 1;                   // z-chunks asked for per problem (at most nz per problem)
    double tuned_ms = 0.0;         // autotuned time of the group's pass (0: not tuned)
    std::vector<int> members;
    void* desc = nullptr;          // BatchProblem<float>[members] in device memory
    double* partials = nullptr;    // 3 doubles per item
    unsigned int* items_done = nullptr;
    unsigned int* work = nullptr;
    int nitems = 0;
    size_t partial_cap = 0;        // items the partials buffer holds
};

}  // namespace

struct bsk_batch {
    int count, prec;
    double dt;
    cudaStream_t stream, cap_stream;
    std::vector<Prob> P;
    std::vector<Group> groups;
    Scalars* sc = nullptr;         // inner (FP32 CG) scalars, one per problem
    Scalars* sc64 = nullptr;       // outer (FP64 residual) scalars, one per problem
    Scalars* gstatus = nullptr;    // wait time-outs of the batched kernels
    Scalars* h_sc = nullptr;       // pinned mirror of count scalars
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    int check_every = 16;          // autotuned graph length
    long long launches = 0;
};

namespace {

int bfail(int code, const char* msg) { return bsk::set_error(code, msg); }

#define BCUDA(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return bfail(BSK_ECUDA, #call " failed");   \
    } while (0)

int build_groups(bsk_batch* B, int timing)
{
    std::vector<char> host(bsk::batch_problem_bytes());
    for (Group& g : B->groups) {
        int item = 0;
        std::vector<char> descs(g.members.size() * bsk::batch_problem_bytes());
        for (size_t i = 0; i < g.members.size(); i++) {
            Prob& p = B->P[g.members[i]];
            double Kdt[3][bsk::kMaxTaps];
            for (int d = 0; d < 3; d++)
                for (int j = 0; j < bsk::kMaxTaps; j++) Kdt[d][j] = B->dt * p.K[d][j];
            int nit = 0;
            BCUDA(bsk::fill_batch_problem(descs.data() + i * bsk::batch_problem_bytes(), g.degree, g.rows, p.nx, p.ny,
                                          p.nz, p.pitch, p.nzc, item, p.M, Kdt, p.r, p.q, p.p, p.x,
                                          B->sc + g.members[i], nullptr, g.items_done + i, timing, &nit));
            item += nit;
        }
        g.nitems = item;
        if ((size_t)item > g.partial_cap) {
            if (g.partials) cudaFree(g.partials);
            g.partials = nullptr;
            cudaError_t e = cudaMalloc((void**)&g.partials, 3 * sizeof(double) * (size_t)item);
            if (e != cudaSuccess) return bfail(BSK_ENOMEM, "batch partials allocation failed");
            g.partial_cap = item;
        }
        // partial-sum slots: problem i uses the slots of its own items
        item = 0;
        for (size_t i = 0; i < g.members.size(); i++) {
            char* d = descs.data() + i * bsk::batch_problem_bytes();
            int nit = 0;
            Prob& p = B->P[g.members[i]];
            double Kdt[3][bsk::kMaxTaps];
            for (int dd = 0; dd < 3; dd++)
                for (int j = 0; j < bsk::kMaxTaps; j++) Kdt[dd][j] = B->dt * p.K[dd][j];
            BCUDA(bsk::fill_batch_problem(d, g.degree, g.rows, p.nx, p.ny, p.nz, p.pitch, p.nzc, item, p.M, Kdt, p.r,
                                          p.q, p.p, p.x, B->sc + g.members[i], g.partials + 3 * (size_t)item,
                                          g.items_done + i, timing, &nit));
            item += nit;
        }
        BCUDA(cudaMemcpyAsync(g.desc, descs.data(), descs.size(), cudaMemcpyHostToDevice, B->stream));
    }
    BCUDA(cudaStreamSynchronize(B->stream));
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return BSK_OK;
}

int enqueue_group(bsk_batch* B, const Group& g, int parity, cudaStream_t s)
{
    bsk::TmaBatchLaunch L;
    L.degree = g.degree;
    L.rows = g.rows;
    L.desc = g.desc;
    L.nprobs = (int)g.members.size();
    L.nitems = g.nitems;
    L.parity = parity;
    L.work = g.work;
    L.status = B->gstatus;
    BCUDA(bsk::launch_tma_batch(L, s));
    return BSK_OK;
}

int enqueue_pass(bsk_batch* B, int parity, cudaStream_t s)
{
    for (Group& g : B->groups)
        if (int rc = enqueue_group(B, g, parity, s)) return rc;
    return BSK_OK;
}

int ensure_graph(bsk_batch* B, int chunk)
{
    if (B->graph && B->graph_chunk == chunk) return BSK_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    BCUDA(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = BSK_OK;
    for (int it = 0; it < chunk && rc == BSK_OK; it++) rc = enqueue_pass(B, it & 1, B->cap_stream);
    cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
    if (rc != BSK_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bfail(BSK_ECUDA, "graph capture failed");
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(BSK_ECUDA, "graph instantiation failed");
    B->graph_chunk = chunk;
    return BSK_OK;
}

int read_scalars(bsk_batch* B, Scalars* dev)
{
    BCUDA(cudaMemcpyAsync(B->h_sc, dev, sizeof(Scalars) * B->count, cudaMemcpyDeviceToHost, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    return BSK_OK;
}

int write_scalars(bsk_batch* B, Scalars* dev)
{
    BCUDA(cudaMemcpyAsync(dev, B->h_sc, sizeof(Scalars) * B->count, cudaMemcpyHostToDevice, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    return BSK_OK;
}

double since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void fill_res(const bsk_batch* B, const Prob& p, bsk::OpLaunch& L, int mode)
{
    memset(&L, 0, sizeof L);
    L.mode = mode;
    L.degree = p.n;
    L.nx = p.nx;
    L.ny = p.ny;
    L.nz = p.nz;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < bsk::kMaxTaps; j++) {
            L.M[d][j] = p.M[d][j];
            L.Kdt[d][j] = B->dt * p.K[d][j];
        }
}

// Lockstep iterative refinement of all problems: FP64 residuals, inner batched FP32 CG.
int batch_solve(bsk_batch* B, const double* const* b, double* const* x, const bsk_cg_opts* opts,
                bsk_cg_report* rep, std::chrono::steady_clock::time_point t0)
{
    const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-8;
    const int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 10000;
    int chunk = (opts && opts->check_every > 0) ? opts->check_every : B->check_every;
    chunk += chunk & 1;
    const double inner_tol = (opts && opts->inner_tol > 0) ? opts->inner_tol : 1e-5;
    const int max_outer = (opts && opts->max_outer > 0) ? opts->max_outer : 30;
    const double tlim = (opts && opts->time_limit_s > 0) ? opts->time_limit_s : 0.0;
    const int n = B->count;
    std::vector<int> active(n, 1), iters(n, 0), outer(n, 0), status(n, BSK_NOT_CONVERGED);
    std::vector<double> rel(n, 0.0);
    int rc = ensure_graph(B, chunk);
    if (rc) return rc;
    for (int k = 0;; k++) {
        // FP64 true residuals of the active problems
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            Prob& p = B->P[i];
            bsk::OpLaunch L;
            fill_res(B, p, L, bsk::MODE_RES);
            L.in0 = x[i];
            L.b = b[i];
            L.out0 = p.r64;
            L.sc = B->sc64 + i;
            L.partials = p.partials64;
            L.fin = bsk::FIN_RES_TRUE;
            BCUDA(bsk::launch_op<double>(L, B->stream));
            B->launches++;
        }
        if ((rc = read_scalars(B, B->sc64))) return rc;
        int left = 0;
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            const double rr = B->h_sc[i].rr_true, bb = B->h_sc[i].bb_true;
            if (!std::isfinite(rr) || !std::isfinite(bb)) { active[i] = 0; status[i] = BSK_EBREAKDOWN; continue; }
            if (bb == 0.0) {
                BCUDA(cudaMemsetAsync(x[i], 0, B->P[i].len * sizeof(double), B->stream));
                active[i] = 0; status[i] = BSK_OK; rel[i] = 0.0; continue;
            }
            rel[i] = std::sqrt(rr / bb);
            if (rel[i] <= tol) { active[i] = 0; status[i] = BSK_OK; continue; }
            if (k >= max_outer || iters[i] >= max_iter) { active[i] = 0; status[i] = BSK_NOT_CONVERGED; continue; }
            left++;
        }
        if (!left) break;
        if (tlim > 0 && since(t0) > tlim) {
            for (int i = 0; i < n; i++)
                if (active[i]) status[i] = BSK_ETIMEOUT;
            break;
        }
        // inner problems: r32 = r64 / ||r64||, x32 = 0, q = p = 0; converged problems stay done
        memset(B->h_sc, 0, sizeof(Scalars) * n);
        for (int i = 0; i < n; i++) {
            Scalars& s = B->h_sc[i];
            if (!active[i]) { s.done = 1; continue; }
            double it = std::max(inner_tol, 0.3 * tol / rel[i]);
            if (it > 0.5) it = 0.5;
            s.tol2 = it * it;
            s.max_iter = std::max(1, max_iter - iters[i]);
        }
        if ((rc = write_scalars(B, B->sc))) return rc;
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            Prob& p = B->P[i];
            k_pack_scaled<<<grid_for(p.plen), 256, 0, B->stream>>>(p.r64, p.r[0], p.nx, p.ny, p.nz, p.pitch,
                                                                  B->sc64 + i);
            BCUDA(cudaGetLastError());
            BCUDA(bsk::launch_cg_init_zero<float>(p.r[0], p.r[0], p.x, p.plen, nullptr, B->sc + i,
                                                  p.partials64, B->stream));
            BCUDA(cudaMemsetAsync(p.q[0], 0, p.plen * sizeof(float), B->stream));
            BCUDA(cudaMemsetAsync(p.p[0], 0, p.plen * sizeof(float), B->stream));
            B->launches += 2;
        }
        for (Group& g : B->groups) BCUDA(cudaMemsetAsync(g.work, 0, 2 * sizeof(unsigned int), B->stream));
        // batched FP32 CG until every inner problem has stopped
        if ((rc = read_scalars(B, B->sc))) return rc;
        for (;;) {
            bool all = true;
            for (int i = 0; i < n; i++) all = all && B->h_sc[i].done;
            if (all) break;
            BCUDA(cudaGraphLaunch(B->graph, B->stream));
            B->launches += (long long)chunk * B->groups.size();
            if ((rc = read_scalars(B, B->sc))) return rc;
            Scalars gs;
            BCUDA(cudaMemcpy(&gs, B->gstatus, sizeof gs, cudaMemcpyDeviceToHost));
            if (gs.status == -4) return bfail(BSK_ETIMEOUT, "a batched kernel timed out waiting for data");
            if (tlim > 0 && since(t0) > tlim) return bfail(BSK_ETIMEOUT, "batch solve exceeded its time limit");
        }
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            iters[i] += B->h_sc[i].iter;
            outer[i] += 1;
            if (B->h_sc[i].status == -5 && B->h_sc[i].iter == 0) { active[i] = 0; status[i] = BSK_EBREAKDOWN; continue; }
            Prob& p = B->P[i];
            k_unpack_update<<<grid_for(p.len), 256, 0, B->stream>>>(x[i], p.x, p.nx, p.ny, p.nz, p.pitch,
                                                                    B->sc64 + i);
            BCUDA(cudaGetLastError());
            B->launches++;
        }
    }
    int worst = BSK_OK;
    for (int i = 0; i < n; i++) {
        if (rep) {
            rep[i].status = status[i];
            rep[i].iterations += iters[i];
            rep[i].outer_iterations += outer[i];
            rep[i].rel_residual = rel[i];
        }
        if (status[i] < 0 && (worst >= 0 || status[i] < worst)) worst = status[i];
        else if (worst >= 0 && status[i] > worst) worst = status[i];
    }
    return worst;
}

}  // namespace

extern "C" int bsk_batch_create(const bsk_problem* probs, int count, int precision, void* stream,
                                bsk_batch** out)
{
    if (!probs || !out || count < 1) return bfail(BSK_EINVAL, "null argument or empty batch");
    *out = nullptr;
    if (precision != BSK_F32_IR) return bfail(BSK_EINVAL, "batches run in BSK_F32_IR");
    const double dt = probs[0].dt;
    for (int i = 0; i < count; i++) {
        const bsk_problem& p = probs[i];
        if (p.degree < 1 || p.degree > 5) return bfail(BSK_EINVAL, "degree outside 1..5");
        if (p.nx < p.degree || p.ny < p.degree || p.nz < p.degree)
            return bfail(BSK_EINVAL, "each axis needs at least degree unknowns");
        if (!(p.hx > 0) || !(p.hy > 0) || !(p.hz > 0)) return bfail(BSK_EINVAL, "grid steps must be > 0");
        if (p.mask) return bfail(BSK_EINVAL, "batched problems are unmasked boxes");
        if (p.dt != dt || !(dt >= 0)) return bfail(BSK_EINVAL, "all problems of a batch share one dt >= 0");
    }
    bsk_batch* B = new (std::nothrow) bsk_batch;
    if (!B) return bfail(BSK_ENOMEM, "host allocation failed");
    B->count = count;
    B->prec = precision;
    B->dt = dt;
    B->stream = (cudaStream_t)stream;
    B->cap_stream = nullptr;
    auto cleanup = [&](int code) {
        bsk_batch_destroy(B);
        return code;
    };
    if (cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(bfail(BSK_ECUDA, "stream creation failed"));
    B->P.resize(count);
    int degrees_present[6] = {0};
    for (int i = 0; i < count; i++) {
        const bsk_problem& q = probs[i];
        Prob& p = B->P[i];
        memset(&p, 0, sizeof p);
        p.nx = q.nx; p.ny = q.ny; p.nz = q.nz; p.n = q.degree;
        p.pitch = (q.nx + 3) / 4 * 4;
        p.h[0] = q.hx; p.h[1] = q.hy; p.h[2] = q.hz;
        p.len = (size_t)q.nx * q.ny * q.nz;
        p.plen = (size_t)p.pitch * q.ny * q.nz;
        p.nzc = 1;
        for (int d = 0; d < 3; d++) bspline_kernels(p.n, p.h[d], p.M[d], p.K[d]);
        degrees_present[p.n] = 1;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 2 && e == cudaSuccess; k++) {
            e = cudaMalloc((void**)&p.r[k], p.plen * 4);
            if (e == cudaSuccess) e = cudaMalloc((void**)&p.q[k], p.plen * 4);
            if (e == cudaSuccess) e = cudaMalloc((void**)&p.p[k], p.plen * 4);
        }
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.x, p.plen * 4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.r64, p.len * 8);
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.b64, p.len * 8);
        const size_t nb = 2 * std::max(bsk::op_grid_blocks(p.nx, p.ny, p.nz, p.n), (size_t)bsk::vec_grid(p.plen));
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.partials64, nb * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cleanup(bfail(BSK_ENOMEM, "batch vector allocation failed"));
        }
        for (float* v : {p.r[0], p.r[1], p.q[0], p.q[1], p.p[0], p.p[1], p.x})
            cudaMemsetAsync(v, 0, p.plen * 4, B->stream);
        if (bsk::prepare_op<double>(p.n) != cudaSuccess || bsk::prepare_op<float>(p.n) != cudaSuccess)
            return cleanup(bfail(BSK_ECUDA, "kernel set-up failed"));
    }
    for (int d = 1; d <= 5; d++) {
        if (!degrees_present[d]) continue;
        if (bsk::batch_grid(d, 3) < 1) return cleanup(bfail(BSK_ECUDA, "batched kernel set-up failed"));
        Group g;
        g.degree = d;
        for (int i = 0; i < count; i++)
            if (B->P[i].n == d) g.members.push_back(i);
        cudaError_t e = cudaMalloc(&g.desc, g.members.size() * bsk::batch_problem_bytes());
        if (e == cudaSuccess) e = cudaMalloc((void**)&g.items_done, g.members.size() * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMalloc((void**)&g.work, 2 * sizeof(unsigned int));
        B->groups.push_back(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cleanup(bfail(BSK_ENOMEM, "batch descriptor allocation failed"));
        }
        cudaMemsetAsync(B->groups.back().items_done, 0, g.members.size() * sizeof(unsigned int), B->stream);
        cudaMemsetAsync(B->groups.back().work, 0, 2 * sizeof(unsigned int), B->stream);
    }
    if (cudaMalloc((void**)&B->sc, sizeof(Scalars) * count) != cudaSuccess ||
        cudaMalloc((void**)&B->sc64, sizeof(Scalars) * count) != cudaSuccess ||
        cudaMalloc((void**)&B->gstatus, sizeof(Scalars)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_sc, sizeof(Scalars) * count) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(bfail(BSK_ENOMEM, "batch scalar allocation failed"));
    }
    cudaMemsetAsync(B->sc, 0, sizeof(Scalars) * count, B->stream);
    cudaMemsetAsync(B->sc64, 0, sizeof(Scalars) * count, B->stream);
    cudaMemsetAsync(B->gstatus, 0, sizeof(Scalars), B->stream);
    if (int rc = build_groups(B, 0)) return cleanup(rc);
    *out = B;
    return BSK_OK;
}

extern "C" void bsk_batch_destroy(bsk_batch* B)
{
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (Prob& p : B->P) {
        for (void* v : {(void*)p.r[0], (void*)p.r[1], (void*)p.q[0], (void*)p.q[1], (void*)p.p[0],
                        (void*)p.p[1], (void*)p.x, (void*)p.r64, (void*)p.b64, (void*)p.partials64})
            if (v) cudaFree(v);
    }
    for (Group& g : B->groups) {
        if (g.desc) cudaFree(g.desc);
        if (g.partials) cudaFree(g.partials);
        if (g.items_done) cudaFree(g.items_done);
        if (g.work) cudaFree(g.work);
    }
    if (B->sc) cudaFree(B->sc);
    if (B->sc64) cudaFree(B->sc64);
    if (B->gstatus) cudaFree(B->gstatus);
    if (B->h_sc) cudaFreeHost(B->h_sc);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    delete B;
}

extern "C" int bsk_batch_cg_solve(bsk_batch* B, const void* const* b, void* const* x,
                                  const bsk_cg_opts* opts, bsk_cg_report* reports)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!B || !b || !x) return bfail(BSK_EINVAL, "null argument");
    for (int i = 0; i < B->count; i++)
        if (!b[i] || !x[i]) return bfail(BSK_EINVAL, "null vector in batch");
    if (reports) memset(reports, 0, sizeof(bsk_cg_report) * B->count);
    B->launches = 0;
    int st = batch_solve(B, (const double* const*)b, (double* const*)x, opts, reports, t0);
    if (reports)
        for (int i = 0; i < B->count; i++) {
            reports[i].elapsed_ms = 1e3 * since(t0);
            reports[i].kernel_launches = B->launches;
        }
    return st;
}

extern "C" int bsk_batch_heat_step(bsk_batch* B, void* const* u, const void* const* q, int nsteps,
                                   const bsk_cg_opts* opts, bsk_cg_report* reports)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!B || !u || nsteps < 0) return bfail(BSK_EINVAL, "bad argument");
    for (int i = 0; i < B->count; i++)
        if (!u[i]) return bfail(BSK_EINVAL, "null vector in batch");
    if (reports) memset(reports, 0, sizeof(bsk_cg_report) * B->count);
    B->launches = 0;
    std::vector<const double*> bs(B->count);
    int st = BSK_OK;
    for (int s = 0; s < nsteps; s++) {
        for (int i = 0; i < B->count; i++) {
            Prob& p = B->P[i];
            bsk::OpLaunch L;
            fill_res(B, p, L, bsk::MODE_MASS);
            L.in0 = u[i];
            L.in1 = q ? q[i] : nullptr;
            L.s = B->dt;
            L.out0 = p.b64;
            L.fin = bsk::FIN_NONE;
            BCUDA(bsk::launch_op<double>(L, B->stream));
            B->launches++;
            bs[i] = p.b64;
        }
        int rs = batch_solve(B, bs.data(), (double* const*)u, opts, reports, t0);
        if (rs < 0) { st = rs; break; }
        if (rs > 0 && st == BSK_OK) st = rs;
    }
    if (reports)
        for (int i = 0; i < B->count; i++) {
            reports[i].elapsed_ms = 1e3 * since(t0);
            reports[i].kernel_launches = B->launches;
        }
    return st;
}

extern "C" int bsk_batch_autotune(bsk_batch* B, int reps, int* check_every_out, double* ms_out)
{
    if (!B || reps < 1) return bfail(BSK_EINVAL, "bad argument");
    // time each degree group's CG pass (finalisers off, no problem stops) for every tile shape and
    // z-chunking, and keep the fastest per group
    memset(B->h_sc, 0, sizeof(Scalars) * B->count);
    int rc = write_scalars(B, B->sc);
    if (rc) return rc;
    static const int rows_cands[] = {2, 3, 4};
    static const int nzc_cands[] = {1, 2, 3, 4, 6, 8};
    const size_t ng = B->groups.size();
    std::vector<double> best_ms(ng, -1.0);
    std::vector<int> best_rows(ng, 3), best_nzc(ng, 1);
    cudaEvent_t e0, e1;
    BCUDA(cudaEventCreate(&e0));
    BCUDA(cudaEventCreate(&e1));
    for (int rows : rows_cands) {
        for (int c : nzc_cands) {
            for (Group& g : B->groups) {
                g.rows = bsk::batch_rows_supported(g.degree, rows) ? rows : 3;
                for (int m : g.members) B->P[m].nzc = std::min(c, B->P[m].nz);
            }
            if ((rc = build_groups(B, 1))) break;
            for (size_t gi = 0; gi < ng && rc == BSK_OK; gi++) {
                Group& g = B->groups[gi];
                if (g.rows != rows) continue;   // this tile shape does not exist for the degree
                BCUDA(cudaMemsetAsync(g.work, 0, 2 * sizeof(unsigned int), B->stream));
                if ((rc = enqueue_group(B, g, 0, B->stream))) break;   // warm-up
                BCUDA(cudaEventRecord(e0, B->stream));
                for (int r = 0; r < reps && rc == BSK_OK; r++) rc = enqueue_group(B, g, r & 1, B->stream);
                BCUDA(cudaEventRecord(e1, B->stream));
                BCUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCUDA(cudaEventElapsedTime(&ms, e0, e1));
                const double per = ms / reps;
                if (best_ms[gi] < 0 || per < best_ms[gi]) {
                    best_ms[gi] = per;
                    best_rows[gi] = rows;
                    best_nzc[gi] = c;
                }
            }
            if (rc) break;
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double total = 0.0;
    for (size_t gi = 0; gi < ng; gi++) {
        Group& g = B->groups[gi];
        g.rows = best_rows[gi];
        g.nzc = best_nzc[gi];
        g.tuned_ms = best_ms[gi];
        for (int m : g.members) B->P[m].nzc = std::min(best_nzc[gi], B->P[m].nz);
        total += best_ms[gi];
    }
    int rc2 = build_groups(B, 0);
    if (rc) return rc;
    if (rc2) return rc2;
    // graph length: longer graphs poll less, shorter ones stop sooner after convergence
    B->check_every = total > 0.5 ? 8 : (total > 0.1 ? 16 : 32);
    if (check_every_out) *check_every_out = B->check_every;
    if (ms_out) *ms_out = total;
    return BSK_OK;
}

extern "C" int bsk_batch_groups(bsk_batch* B, int cap, int* degree, int* tile_rows, int* nzc, double* ms)
{
    if (!B || cap < 0) return bfail(BSK_EINVAL, "bad argument");
    const int ng = (int)B->groups.size();
    for (int gi = 0; gi < ng && gi < cap; gi++) {
        const Group& g = B->groups[gi];
        if (degree) degree[gi] = g.degree;
        if (tile_rows) tile_rows[gi] = 8 * g.rows;
        if (nzc) nzc[gi] = g.nzc;
        if (ms) ms[gi] = g.tuned_ms;
    }
    return ng;
}

extern "C" int bsk_batch_configure(bsk_batch* B, int degree, int tile_rows, int nzc, int check_every)
{
    if (!B || nzc < 1 || check_every < 1 || tile_rows % 8 != 0) return bfail(BSK_EINVAL, "bad argument");
    const int rows = tile_rows / 8;
    bool any = false;
    for (Group& g : B->groups) {
        if (degree != 0 && g.degree != degree) continue;
        if (!bsk::batch_rows_supported(g.degree, rows)) return bfail(BSK_EINVAL, "tile shape not available for this degree");
        if (bsk::batch_grid(g.degree, rows) < 1) return bfail(BSK_ECUDA, "batched kernel set-up failed");
        g.rows = rows;
        g.nzc = nzc;
        g.tuned_ms = 0.0;
        for (int m : g.members) B->P[m].nzc = std::min(nzc, B->P[m].nz);
        any = true;
    }
    if (!any) return bfail(BSK_EINVAL, "no group of that degree");
    B->check_every = check_every + (check_every & 1);
    return build_groups(B, 0);
}
