// bsk_launch.h -- host-side launch interface between the C ABI (bsk_api.cu) and the kernel
// translation units (one per element type).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <chrono>
#include <functional>

#include "bsk_device.cuh"

struct bsk_net;

namespace bsk {

// Records msg as the calling thread's last error (read back by bsk_last_error) and returns code.
int set_error(int code, const char* msg);

struct OpLaunch {
    int mode;                    // OpMode
    int degree;                  // 1..5
    int nx, ny, nz;
    const uint8_t* mask;         // device node mask or nullptr
    double M[3][kMaxTaps];       // per-axis mass kernels (axis 0 = x)
    double Kdt[3][kMaxTaps];     // per-axis stiffness kernels, multiplied by dt
    const void* in0;
    const void* in1;
    void* out0;
    void* out1;
    void* xvec;
    const void* b;
    double s;
    Scalars* sc;
    double* partials;
    int fin;
    int p_parity;
    int bf16io;                  // FP32 kernels, MODE_OP / MODE_MASS: in0, in1, out0 hold bfloat16
    // Variable coefficients (op_var.cuh): nodal fields D and mu_a at the (nz+2)(ny+2)(nx+2) nodes,
    // as float [0] and double [1]; null = the constant-coefficient operator. MODE_MASS ignores them.
    const void* vd[2];
    const void* vm[2];
    double h[3];                 // grid steps (variable-coefficient tables)
    double dt;                   // weight of the diffusion term (variable coefficients)
    // Robin problems: band rows near the faces (op_generic.cuh, robin_row), float [0] / double
    // [1]; null = odd reflection at the faces
    const void* rb[2];
    // MODE_CGP: Jacobi diagonal factors (op_generic.cuh, jacobi_inv), float [0] / double [1];
    // null = no preconditioner
    const void* jac[2];
    int jn;                      // row length of the jac tables
    // MODE_CGP: 1 / diag A per node (Jacobi), float [0] / double [1]; the kernels read it instead
    // of the jac tables; null = no preconditioner
    const void* jvec[2];
    // MODE_OP on a z-slab (Geom): global offset, global plane count (0 = nz: a whole grid) and
    // the halo planes in0 carries on each side
    int z_off, nz_glob, zpad;
};

// Grid of the operator kernel for a problem; partial-sum buffers hold 2 doubles per block.
dim3 op_grid(int nx, int ny, int nz, int degree, int* tz);
size_t op_grid_blocks(int nx, int ny, int nz, int degree);
int vec_grid(size_t len);

// One-time per-process set-up of the operator kernels of one degree (shared-memory limits);
// called by bsk_create, never inside a stream capture.
template <typename T>
cudaError_t prepare_op(int degree);

template <typename T>
cudaError_t launch_op(const OpLaunch& L, cudaStream_t s);

// Variable-coefficient operator (op_var.cuh, var_impl.cuh): MODE_OP, MODE_RES, MODE_CGP with the
// fields L.vd / L.vm of the element type.
template <typename T>
cudaError_t launch_var(const OpLaunch& L, cudaStream_t s);
template <typename T>
cudaError_t prepare_var(int degree);
template <typename T>
size_t var_grid_blocks(int nx, int ny, int nz, int degree);
// Floating-point operations the variable-coefficient kernel executes per node (halo included).
template <typename T>
double var_flops_per_node(int degree, int nx, int ny, int nz);
// dst = src (converted), or 1 everywhere when src is null.
template <typename T>
cudaError_t launch_coef_fill(const double* src, T* dst, size_t len, cudaStream_t s);

template <typename T>
cudaError_t launch_cg_update(T* r, const T* q, size_t len, Scalars* sc, double* partials,
                             int fin, cudaStream_t s);
// Jacobi-preconditioned CG (vec_kernels.cuh): r -= alpha q with r.r and r.z (FIN_UPD_PC), and
// the starting r.z (FIN_PC_INIT).
// The inverse diagonal is jvec[i] when jvec is given, else formed from the per-axis tables jac.
template <typename T>
cudaError_t launch_cg_update_pc(T* r, const T* q, size_t len, int nx, int ny, const T* jac, int jn, const T* jvec,
                                Scalars* sc, double* partials, int fin, cudaStream_t s);
template <typename T>
cudaError_t launch_pc_dot(const T* r, size_t len, int nx, int ny, const T* jac, int jn, const T* jvec,
                          Scalars* sc, double* partials, cudaStream_t s);
// jinv[i] = 1 / diag A of the separable operator at flat index i, from the per-axis tables jac
// (vec_kernels.cuh, k_jacobi_fill).
template <typename T>
cudaError_t launch_jacobi_fill(T* jinv, size_t len, int nx, int ny, const T* jac, int jn, cudaStream_t s);
// Diagonal probing (var_impl.cuh): take = 0 fills v with the indicator of colour (cx, cy, cz)
// modulo stride; take = 1 stores 1 / y at that colour's nodes into jinv.
template <typename T>
cudaError_t launch_probe(T* v, const T* y, T* jinv, int take, int nx, int ny, int nz, int stride, int cx,
                         int cy, int cz, const uint8_t* mask, cudaStream_t s);
// Element type conversions (transform.cu).
cudaError_t launch_convert_f32_f64(const float* src, double* dst, size_t len, cudaStream_t s);
cudaError_t launch_convert_f64_f32(const double* src, float* dst, size_t len, cudaStream_t s);
// Banded transfer along one axis (transform.cu): out[.., f, ..] = sum_k T[f][k] in[.., c0[f] + k, ..]
// for f < nout, the other two extents unchanged (dims are those of `in`, x fastest).
template <typename T>
cudaError_t launch_transfer(const T* in, T* out, int nx, int ny, int nz, int axis, int nout, int w,
                            const T* tab, const int* c0, cudaStream_t s);

template <typename T>
cudaError_t launch_cg_flush(T* x, const T* p0, const T* p1, size_t len, const Scalars* sc,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_cg_init_zero(const T* b, T* r, T* x, size_t len, const uint8_t* mask,
                                Scalars* sc, double* partials, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_masked(const T* src, T* dst, size_t len, const uint8_t* mask,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_norm2(const T* x, size_t len, Scalars* sc, double* partials, cudaStream_t s);

// ---- TMA operator kernels (op_tma.cuh): unmasked problems with 16-byte row pitch ----
struct TmaLaunch {
    int mode;                    // TMODE_OP, TMODE_RES or TMODE_CG
    int degree;
    int nx, ny, nz;
    double M[3][kMaxTaps];
    double Kdt[3][kMaxTaps];
    const void* in[3];           // OP/RES: {x}; CG: {p_{m-1}, q_{m-1}, p_{m-2}} (no r is kept)
    const void* inint;           // RES: b; CG: x
    void* out0;                  // OP y; RES r; CG q_m
    void* out1;                  // unused
    void* out2;                  // CG p_m
    void* xvec;                  // CG x (in place)
    const uint8_t* mask;         // node mask or null (outputs zeroed where 0; inputs must be)
    const uint32_t* mbits;       // the same mask bit-packed (launch_pack_mask); required with mask
    const uint8_t* occ;          // tile occupancy per plane (tile_occupancy), null without a mask
    Scalars* sc;
    double* partials;            // 3 doubles per block of the resident grid
    unsigned int* work;          // 2 counters, zero between launches (dynamic item queue)
    int fin;
    int impl;                    // TMODE_CG, FP32, unmasked, degree <= 4: 0 = the warp-specialised
                                 // pass (op_ws.cuh), 1 = the single-pass kernel of op_tma.cuh
    int ws_chunk;                // warp-specialised CG pass: most planes per z-chunk (0 = 128)
    // TMODE_OP on a z-slab: global offset, global plane count (0 = nz) and the halo planes in[0]
    // carries on each side (0 = a whole grid)
    int z_off, nz_glob, zpad;
};
// In-place banded triangular solves along one axis (0 = x, 1 = y, 2 = z) of an nx*ny*nz grid,
// one thread per line: L holds a banded Cholesky factor of half-width p <= 5 (transform.cu).
template <typename T>
cudaError_t launch_band_solve(T* d, int nx, int ny, int nz, int axis, int p, const T* L, cudaStream_t s);

// occ[z * tiles + tile] = 1 iff the 64 x 24 tile (x fastest) has an active node in plane z.
cudaError_t launch_tile_occupancy(const uint8_t* mask, int nx, int ny, int nz, uint8_t* occ, cudaStream_t s);
// Bit-packed copy of a node mask for the TMA kernels: mask_words(nx) 32-bit words per
// (z, y) row, bit i of word w = node x = 32 w + i (tma_f32.cu).
int mask_words(int nx);
cudaError_t launch_pack_mask(const uint8_t* mask, int nx, int ny, int nz, uint32_t* bits, cudaStream_t s);
int tma_tiles(int nx, int ny);
struct dfl;   // double-float element (dfloat.cuh): the FP64-accurate residual on the FP32 pipes
template <typename T>
int tma_max_degree();
template <typename T>
cudaError_t prepare_tma(int degree);
template <typename T>
int tma_grid(int degree, int mode);   // resident blocks (after prepare_tma), 0 if unsupported
template <typename T>
cudaError_t launch_tma(const TmaLaunch& L, cudaStream_t s);

// Warp-specialised FP32 passes (op_ws.cuh): unmasked y = A x and the single-pass CG iteration,
// degrees 1..4; launch_tma<float> takes them for TMODE_OP and TMODE_CG without a mask.
// prepare_ws is called by prepare_tma<float>.
bool ws_supported(int degree);
cudaError_t prepare_ws(int degree);
cudaError_t launch_ws(const TmaLaunch& L, cudaStream_t s);

// Batched single-pass CG iteration (FP32): one persistent launch over the items of all the
// problems of one degree; desc points to BatchProblem<float>[nprobs] in device memory.
struct TmaBatchLaunch {
    int degree;
    int rows;                    // output rows per warp of the tile (tile = 64 x 8 rows): 2, 3 or 4
    const void* desc;
    int nprobs;
    int nitems;
    int parity;
    unsigned int* work;          // 2 counters, zero between launches
    Scalars* status;             // receives a wait time-out
};
// Highest degree with a 64 x 32 batched tile (its accumulators would spill above it).
constexpr int kBatchMaxDegreeR4 = 4;
size_t batch_problem_bytes();
bool batch_rows_supported(int degree, int rows);
int batch_grid(int degree, int rows);   // resident blocks of the batched kernel (0 if unsupported)
// Fills one BatchProblem<float> (host memory, batch_problem_bytes() bytes) for a padded problem
// cut into tiles of 64 x 8 rows and nzc z-chunks.
cudaError_t fill_batch_problem(void* host_desc, int degree, int rows, int nx, int ny, int nz, int pitch,
                               int nzc, int item0, const double (*M)[kMaxTaps],
                               const double (*Kdt)[kMaxTaps], float* const r[2], float* const q[2],
                               float* const p[2], float* x, Scalars* sc, double* partials,
                               unsigned int* items_done, int timing, int* nitems_out);
cudaError_t launch_tma_batch(const TmaBatchLaunch& L, cudaStream_t s);

// ---- flexible CG with the learned preconditioner (fcg.cu, net.cu) ----
struct FcgVectors {
    const float* b;      // right-hand side of the inner solve
    float *x, *r, *p, *q, *z, *rn, *zn;
    double* partials;    // 3 doubles per block of the vector kernels (1216 blocks at most)
    void* state;         // fcg_state_bytes()
    // optional record of the iteration (fcg_record): before iteration k < rec_steps, r and x
    // are copied to rec_r + k n and rec_x + k n; null = no record
    float* rec_r;
    float* rec_x;
    int rec_steps;
};
size_t fcg_state_bytes();
// The network maps r linearly (BSK_ACT_LINEAR): N(r / ||r||) ||r|| = N(r), no normalisation.
bool net_linear(const bsk_net* net);
int fcg_inner(const FcgVectors& V, size_t n, const uint8_t* mask, double tol, int max_iter, int stall_window,
              double out_scale, double jac, const std::function<int(const float*, float*)>& op, bsk_net* net,
              const std::function<int(bsk_net*, const float*, const uint8_t*, float*)>& net_forward,
              cudaStream_t s, int* iters, int* fallback_iter, int* rejected, double time_limit,
              std::chrono::steady_clock::time_point t0);

// ---- CG vector passes of a z-slab (slab.cu); s is the BSK_SLAB_* scalar array ----
enum SlabPass { SLAB_BEGIN, SLAB_DOT, SLAB_UPDATE, SLAB_FIRST, SLAB_DIRECTION };
struct SlabVectors {
    const void *b, *ax, *q;   // local planes
    void *x, *r, *p;          // local planes (p: the first local plane of the halo array)
};
template <typename T>
cudaError_t slab_pass(int pass, const SlabVectors& v, size_t len, double* s, double* partials, unsigned* ctr,
                      cudaStream_t st);
size_t slab_partials_doubles();

cudaError_t launch_ir_scale_down(const double* r64, float* r32, size_t len, const Scalars* outer,
                                 cudaStream_t s);
cudaError_t launch_ir_update(double* x64, const float* d32, size_t len, const Scalars* outer,
                             cudaStream_t s);

}  // namespace bsk
