/*
 * bsk.h -- C ABI of the GB300 tensor B-spline heat-equation library.
 *
 * The library applies, matrix-free, the Galerkin operator of one implicit Euler step of the heat
 * equation discretised with degree-n tensor B-splines on a uniform grid,
 *
 *     A = Mz (x) My (x) Mx  +  dt ( Kz (x) My (x) Mx + Mz (x) Ky (x) Mx + Mz (x) My (x) Kx ),
 *
 * and solves A x = b with conjugate gradients (paper arXiv:1904.03057: Eq. RitzGalerkin and
 * Eq. tensForm with constant coefficients D = dt, mu_a = 1; the separable shift-invariant
 * kernels of section 2.4 and the filtering algorithm of Fig. FiltAlg; the CG stage of
 * section 2.5). Md and Kd are the (2n+1)-tap mass and stiffness kernels of axis d,
 * Md = hd * beta^{2n+1}(j) and Kd = -(1/hd) * (beta^{2n-1}(j+1) - 2 beta^{2n-1}(j) +
 * beta^{2n-1}(j-1)), j = -n..n (scalar-product and derivative identities, Table tblBsplines).
 * A handle can instead carry variable coefficients D(x), mu_a(x) expanded in B-splines
 * (bsk_set_coefficients: the operator of Eq. tensForm computed on the fly), the boundary
 * penalty of the paper's large run over the untruncated basis (bsk_set_boundary), and the
 * Jacobi preconditioner (bsk_set_preconditioner); bsk_prolong starts a fine Robin solve from a
 * coarse one, bsk_transform maps between B-spline coefficients and node values, and a learned
 * preconditioner drives flexible CG (fcg_solve).
 *
 * Conventions shared by every entry point (the Robin boundary changes the second; see
 * bsk_set_boundary):
 *   - Arrays are dense, x fastest: element (k, j, i) of an nx*ny*nz grid sits at
 *     ((k * ny) + j) * nx + i. Unknown i of an axis is the B-spline centred at (i + 1) h.
 *   - Zero Dirichlet data on the box faces: coefficients are odd-reflected about the faces,
 *     which sit one grid step beyond the first and the last unknown (positions 0 and
 *     (N + 1) h), where the coefficient is zero. This needs N >= n unknowns per axis.
 *   - An optional node mask selects the active unknowns (1 = active). Inactive unknowns are
 *     removed from the system: they read as zero and are written as zero.
 *   - Every vector argument is a DEVICE pointer owned by the caller, with the element type of
 *     the handle's precision (see bsk_create). Input and output vectors must not overlap.
 *   - All work is enqueued on the handle's CUDA stream. Entry points that report results
 *     (cg_solve, heat_step) synchronise that stream before returning; op_apply and mass_apply
 *     return as soon as the work is enqueued.
 *   - Functions return a status code: 0 on success, > 0 for soft outcomes, < 0 for errors.
 *     Errors never abort the process and never trap the GPU; bsk_last_error() describes the
 *     most recent error of the calling thread.
 */
#ifndef BSK_H
#define BSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define BSK_OK 0
#define BSK_NOT_CONVERGED 1   /* max_iter reached before the tolerance                       */
#define BSK_STALLED 2         /* residual stopped decreasing (stall window exceeded)          */
#define BSK_EINVAL (-1)       /* invalid argument (null pointer, size, degree, overlap, ...)  */
#define BSK_ECUDA (-2)        /* a CUDA runtime call failed                                   */
#define BSK_ENOMEM (-3)       /* device or host allocation failed                             */
#define BSK_ETIMEOUT (-4)     /* a wall-clock limit was exceeded: the solve's time limit, or a
                                 bounded device wait of the network (bsk_net_read_loss)      */
#define BSK_EBREAKDOWN (-5)   /* CG breakdown: p.Ap <= 0, or a NaN/Inf in a reduction         */

/* ---- precision modes --------------------------------------------------------------------- */
#define BSK_F64 0     /* vectors double; operator and reductions in FP64                         */
#define BSK_F32 1     /* vectors float; operator in FP32; CG scalars and reductions in FP64       */
#define BSK_F32_IR 2  /* vectors double; FP64-accurate true residual b - A x (double-float
                         arithmetic where the grid allows, see bsk_residual) and FP64 update of
                         x around an inner FP32 CG (iterative refinement); CG scalars in FP64     */
#define BSK_BF16S 3   /* BF16 storage: op_apply / mass_apply only, vectors bfloat16 (uint16 bit
                         patterns), arithmetic FP32, each output rounded to nearest BF16 once.
                         An operator variant for measuring what BF16 storage costs in accuracy
                         (at most 2^-8 relative per stored value); the solvers reject it         */

/* Galerkin kernels of degree-n B-splines on a grid of step h (Table tblBsplines, scalar-product
 * and derivative rows):
 *   mass[j + n]  = h * beta^{2n+1}(j),
 *   stiff[j + n] = -(1/h) * (beta^{2n-1}(j+1) - 2 beta^{2n-1}(j) + beta^{2n-1}(j-1)),
 * j = -n..n. mass and stiff are HOST arrays of 2n+1 doubles owned by the caller. The values are
 * exact rationals (integer numerators over (2n+1)! and (2n-1)!) rounded once to double, then
 * scaled by h or 1/h. Returns BSK_EINVAL for n < 1, n > 5, h <= 0 (or NaN) or a null pointer. */
int bspline_kernels(int n, double h, double* mass, double* stiff);

/* A heat problem on a box grid. */
typedef struct bsk_problem {
    int nx, ny, nz;        /* unknowns per axis, each >= degree                                 */
    int degree;            /* B-spline degree n, 1..5                                           */
    double hx, hy, hz;     /* grid steps (> 0); the library does not assume hd = 1/(Nd + 1)     */
    double dt;             /* implicit Euler time step, the weight of the stiffness term (>= 0) */
    const uint8_t* mask;   /* DEVICE pointer to nz*ny*nx bytes (non-zero = active), or NULL for
                              the whole box. Copied at bsk_create; the caller keeps ownership.  */
} bsk_problem;

typedef struct bsk_handle bsk_handle;

/* Creates a solver handle for the implicit-Euler system of one box (Eq. tensForm, section 2.4:
 * A = Mz (x) My (x) Mx + dt (Kz (x) My (x) Mx + Mz (x) Ky (x) Mx + Mz (x) My (x) Kx) with the
 * kernels of Table tblBsplines; with a mask, its principal submatrix on the active nodes).
 * It validates the problem, uploads the kernels and the mask, allocates
 * every work vector the handle needs for op_apply, mass_apply, cg_solve and heat_step (the hot
 * loop never allocates), and binds the handle to `stream` (a cudaStream_t; NULL = the legacy
 * default stream). precision is BSK_F64, BSK_F32, BSK_F32_IR or BSK_BF16S (operator only, no
 * work vectors; cg_solve, heat_step and fcg_solve return BSK_EINVAL). On success *out receives
 * the handle, to be released with bsk_destroy. */
int bsk_create(const bsk_problem* prob, int precision, void* stream, bsk_handle** out);

/* Releases the handle and its device memory (after synchronising its stream). NULL is a no-op. */
void bsk_destroy(bsk_handle* h);

/* Changes dt, the weight of the stiffness term in the implicit-Euler operator (Eq. tensForm),
 * of an existing handle. The Robin rows and the Jacobi diagonal of the handle, which carry dt,
 * are rebuilt. */
int bsk_set_dt(bsk_handle* h, double dt);

/* y = A x: the full operator, three axis sweeps fused in one pass (Fig. FiltAlg). x and y are
 * device vectors of nx*ny*nz elements of the handle's element type. */
int op_apply(bsk_handle* h, const void* x, void* y);

/* y = (Mz (x) My (x) Mx) x: the mass operator alone (the mass chain of Fig. FiltAlg). */
int mass_apply(bsk_handle* h, const void* x, void* y);

/* Options of the iterative solvers. Zero-initialise and set what is needed; zero fields take
 * the defaults given in brackets. */
typedef struct bsk_cg_opts {
    double tol;            /* stop when ||r|| <= tol ||b|| [1e-8]                                */
    int max_iter;          /* CG iterations (inner iterations summed, in BSK_F32_IR) [10000]     */
    int check_every;       /* iterations per device-side chunk between host polls, rounded up
                              to a multiple of 6 [16 -> 18]                                      */
    int stall_window;      /* stop with BSK_STALLED when ||r|| has not reached a new minimum for
                              this many iterations [0 = off]                                     */
    double inner_tol;      /* BSK_F32_IR: relative tolerance of each inner FP32 solve [1e-5]    */
    int max_outer;         /* BSK_F32_IR: refinement steps [30]                                 */
    double time_limit_s;   /* wall-clock limit of one call [0 = none]                            */
    int residual_fp64;     /* BSK_F32_IR: 1 = evaluate the true residual b - A x in FP64
                              arithmetic; 0 = double-float arithmetic on the FP32 pipes where
                              the grid allows it (bsk_residual), the default                    */
} bsk_cg_opts;

/* What a solve did. */
typedef struct bsk_cg_report {
    int status;            /* the returned status                                               */
    int iterations;        /* CG iterations (all inner iterations in BSK_F32_IR)                */
    int outer_iterations;  /* refinement steps (BSK_F32_IR), else 0                              */
    double rel_residual;   /* true ||b - A x|| / ||b||, recomputed from x after the solve, in the
                              handle's operator precision (FP64 for BSK_F64 and BSK_F32_IR)      */
    double elapsed_ms;     /* wall-clock time of the call                                        */
    long long kernel_launches; /* kernels this call launched on the GPU (graph nodes included) */
    int fallback_iter;     /* fcg_solve: inner iteration at which the last inner solve fell back
                              to plain CG, -1 if it never did; 0 for the other solvers            */
    int net_rejected;      /* fcg_solve: iterations whose network direction was replaced by r   */
    double iter_ms;        /* cg_solve / heat_step: device time (CUDA events on the handle's
                              stream) from the first to the end of the last CUDA-graph launch of
                              the CG iterations, summed over the inner solves; iter_ms divided by
                              the iterations bounds the time of one iteration's kernel from above
                              (the few launches that find the solve done add to it). 0 for
                              fcg_solve and the batch solvers.                                    */
    double h2d_ms;         /* heat_step_host: device time of the host -> device copies; else 0   */
    double d2h_ms;         /* heat_step_host: device time of the device -> host copy; else 0     */
} bsk_cg_report;

/* Solves A x = b by conjugate gradients (section 2.5), starting from the x passed in, which
 * receives the solution. The operator application, the p.Ap and r.r reductions and the vector
 * updates run on the device; the host only polls a status word every check_every iterations.
 * opts and report may be NULL. Returns BSK_OK, BSK_NOT_CONVERGED, BSK_STALLED or an error. */
int cg_solve(bsk_handle* h, const void* b, void* x, const bsk_cg_opts* opts, bsk_cg_report* report);

/* nsteps implicit Euler steps of u_t = Laplace(u) + g with zero Dirichlet faces:
 * (M + dt K) u^{k+1} = M (u^k + dt q), each solved by cg_solve from u^k. u (in/out) holds the
 * B-spline coefficients; q (may be NULL) the coefficients of the time-constant source g
 * (Eq. RitzGalerkin right-hand side with the source in the same basis). report (may be NULL)
 * sums the iterations over the steps and gives the last step's residual. */
int heat_step(bsk_handle* h, void* u, const void* q, int nsteps, const bsk_cg_opts* opts,
              bsk_cg_report* report);

/* Device-side sum of squares of a handle vector (FP64 accumulation); *out is written on the
 * host after synchronising the stream. Used to check results without a host copy. */
int bsk_norm2(bsk_handle* h, const void* x, double* out);

/* B-spline transforms at the grid nodes (section 2.3, Fig. figBspnSignProc), on the handle's
 * grid and degree, over the whole box (the mask is not applied):
 *   BSK_TO_SAMPLES  out = u, the values sum_i c_i psi_i(x_j) of the coefficients in = c at the
 *                   nodes x_j (indirect transform): a separable convolution with the sampled
 *                   B-spline beta^n(j), odd-reflected at the faces like the operator;
 *   BSK_TO_COEFFS   out = c, the coefficients whose indirect transform is in = f (direct
 *                   transform by interpolation): per axis the band system of the sampled
 *                   basis (positive definite, half-width ceil((n+1)/2) - 1) is solved along every
 *                   grid line with its Cholesky factor (computed and kept by the first call).
 * in, out: DEVICE vectors of the handle's element type (float for BSK_F32, double otherwise),
 * not overlapping. Enqueued on the handle's stream; returns without synchronising.
 * BSK_BF16S handles and unknown directions give BSK_EINVAL. */
#define BSK_TO_SAMPLES 0
#define BSK_TO_COEFFS 1
int bsk_transform(bsk_handle* h, int direction, const void* in, void* out);

/* r = b - A x with the handle's true-residual kernel, and ||r||^2, ||b||^2 (FP64, written on the
 * host after the stream is synchronised; either pointer may be NULL). b, x, r: DEVICE vectors of
 * the handle's element type; entries of b off the mask are ignored, x must be zero there.
 * BSK_F32_IR handles evaluate A x in double-float arithmetic (hi + lo float pairs, exact
 * products and two-sums: about 2^-44 relative per operation, so r agrees with an FP64
 * evaluation to about 1e-13 of the |A||x| scale) on the FP32 pipes when the grid takes the TMA
 * kernels (16-byte rows, degree <= 3); fp64 != 0 forces FP64 arithmetic. This is the residual the
 * refinement of cg_solve / heat_step / fcg_solve uses. */
int bsk_residual(bsk_handle* h, const void* b, const void* x, void* r, int fp64, double* rr, double* bb);

/* Variable coefficients (Eq. RitzGalerkin and Eq. tensForm, section 2.3: the diffusion D(x) and
 * the absorption mu_a(x) expanded in the same B-splines as the solution). After this call the
 * handle's operator is
 *   (A x)_l = sum_k sum_m x_k ( dt d_m w^{klm} + m_m f^{klm} )
 *           = integral of dt D grad psi_l . grad u + mu_a psi_l u,   u = sum_k x_k psi_k,
 * with D = sum_m d_m beta_m, mu_a = sum_m m_m beta_m: for the heat equation
 * u_t = div(D grad u) - mu_a u + g one implicit Euler step takes m = 1 + dt mu_a. d = m = 1
 * gives back the constant-coefficient operator M + dt K. The operator is computed on the fly
 * (strategy (c) of section 2.4) by exact Gauss quadrature per knot interval with sum
 * factorisation, in the handle's CG precision, and every solver and residual of the handle uses
 * it (heat_step keeps the constant mass matrix for its right-hand side M (u + dt q)).
 *   d, m: DEVICE arrays of (nz+2)*(ny+2)*(nx+2) doubles, x fastest: the coefficients at the
 *         nodes 0..N+1 of each axis, box faces included (unknown i sits at node i + 1). Beyond
 *         the faces they are extended evenly (node -e takes node e's value), so that D and mu_a
 *         are even about each face. Either may be NULL, meaning 1 everywhere; both NULL returns
 *         the handle to the constant-coefficient operator. The fields are copied (converted to
 *         FP32 for FP32 passes); the caller keeps ownership of d and m.
 * Synchronises the handle's stream. BSK_BF16S handles give BSK_EINVAL; BSK_ENOMEM if the copies
 * cannot be allocated. */
int bsk_set_coefficients(bsk_handle* h, const double* d, const double* m);

/* Boundary treatment (Eq. RitzGalerkin, section 2.3; the boundary penalty method of section 3).
 *   BSK_BC_DIRICHLET  (default) zero Dirichlet faces: the B-splines odd-reflected at the faces
 *                     (they vanish there); unknown i sits at node i + 1 of an axis of nx + 2 nodes.
 *   BSK_BC_ROBIN      the boundary penalty method: the untruncated B-splines, every beta(x/h - i)
 *                     whose support meets the box, with the integrals truncated to the box and
 *                     the boundary term penalty * integral over the faces of phi psi ds added:
 *                       A = M + dt K + penalty E,  E = sum over faces of (face values outer
 *                       product) x (the other two axes' mass),
 *                     which approximates zero Dirichlet data as penalty grows (the paper's
 *                     1/(2 gamma)). The handle's nx, ny, nz are then the UNKNOWNS per axis: for a box
 *                     of N interior nodes (h = box length / (N + 1)) that is N + 2 + 2 floor(n/2),
 *                     unknown a being the B-spline centred at (a - floor(n/2)) h; every vector of
 *                     the handle has nx*ny*nz entries in that order. Needs no mask, constant
 *                     coefficients, and at least 2 (n + 1) unknowns per axis.
 * The untruncated basis is ill-conditioned for n >= 2 (the outermost B-splines meet the box in a
 * short interval), and more so for large penalties: the Jacobi preconditioner offsets the first
 * part. Synchronises the handle's stream. BSK_EINVAL on an unknown kind, a negative or
 * non-finite penalty, or a handle that does not meet the conditions above. bsk_transform takes
 * Dirichlet handles only. */
#define BSK_BC_DIRICHLET 0
#define BSK_BC_ROBIN 1
int bsk_set_boundary(bsk_handle* h, int kind, double penalty);

/* Preconditioner of the handle's CG solves (cg_solve, heat_step, and the inner solves of
 * BSK_F32_IR refinement):
 *   BSK_PC_NONE    plain CG (default);
 *   BSK_PC_JACOBI  Jacobi-preconditioned CG, z = r / diag(A) (the solver of the paper's large run,
 *                  section 3). The handle keeps 1 / diag(A) per node, one vector in the CG
 *                  precision. With constant coefficients it is formed from the per-axis diagonals
 *                  of the separable operator (with the reflection terms of the Dirichlet basis, or
 *                  the Robin rows). With variable coefficients it is computed by probing:
 *                  (n + 1)^3 operator applications to the indicator vectors of the node classes
 *                  congruent modulo n + 1 per axis. Either is redone when the coefficients, dt or
 *                  the boundary change. The CG iteration then takes the two-pass general kernels.
 * Synchronises the stream; BSK_ENOMEM if the per-node diagonal cannot be allocated. */
#define BSK_PC_NONE 0
#define BSK_PC_JACOBI 1
int bsk_set_preconditioner(bsk_handle* h, int kind);

/* Coarse-grid initialisation (section 3: the large run starts from a solution computed on a
 * grid five times coarser): xf = the L2 projection onto the fine handle's Robin basis of the
 * function sum_c xc_c beta_c of the coarse handle's Robin basis. Both handles: BSK_BC_ROBIN, the
 * same degree and element type, grids covering the same box (box length = (nx - 1 - 2 floor(n/2)) h
 * per axis, equal to 1e-12). Per axis the projection is M_f^{-1} T with T_fc the integral over the
 * box of the product of a fine and a coarse B-spline (exact Gauss quadrature between the
 * breakpoints of both grids) and M_f the fine Gram matrix (banded Cholesky), applied as three
 * banded transfer passes and three passes of line solves. Where the coarse space lies in the fine
 * one (odd degree, coarse step a multiple of the fine step) the function is reproduced exactly.
 * xc: DEVICE vector of the coarse handle's size, xf: of the fine handle's (not overlapping).
 * FP32 handles compute in FP64 internally (temporary FP64 copies; the untruncated Gram matrices
 * are ill-conditioned for n >= 2) and round the result once. Runs on the fine handle's stream and
 * returns after it is synchronised. */
int bsk_prolong(bsk_handle* fine, bsk_handle* coarse, const void* xc, void* xf);

/* Floating-point operations per grid node of one operator application (FMA = 2): the
 * algorithmic count of the method as implemented (the seven band convolutions of Fig. FiltAlg
 * for constant coefficients; the per-cell Gauss quadrature with sum factorisation, without
 * block-halo recomputation, for variable coefficients) and the count the kernel executes on this
 * grid, recomputed halo cells included. Either pointer may be NULL. */
int bsk_op_flops(bsk_handle* h, double* algorithmic, double* executed);

/* ---- batches of independent problems ------------------------------------------------------
 * Many unmasked box problems (any sizes, degrees 1..5, one shared dt) solved together: each CG
 * iteration of the whole batch is one persistent launch per degree present, whose blocks take
 * (problem, tile, z-chunk) work items from a device queue; every problem keeps its own CG
 * scalars and convergence test and leaves the queue once converged. Inner iterations run in
 * FP32 inside CUDA graphs; each problem's true residual and update are FP64 (iterative
 * refinement, precision must be BSK_F32_IR). The batch owns its work vectors (row-padded FP32
 * copies plus FP64 residuals), allocated at creation. */
typedef struct bsk_batch bsk_batch;

/* probs: HOST array of `count` problems (mask must be NULL; all dt equal). */
int bsk_batch_create(const bsk_problem* probs, int count, int precision, void* stream, bsk_batch** out);
void bsk_batch_destroy(bsk_batch* b);

/* CG (section 2.5) on every problem's system A x = b (Eq. tensForm), inside iterative
 * refinement. b, x: HOST arrays of `count` DEVICE pointers to dense double vectors (x in: start, out:
 * solution). reports (may be NULL): HOST array of `count` reports. The returned status is the
 * worst of the problems' statuses. opts as for cg_solve (applied to every problem). */
int bsk_batch_cg_solve(bsk_batch* b, const void* const* bvec, void* const* x, const bsk_cg_opts* opts,
                       bsk_cg_report* reports);

/* nsteps implicit Euler steps of every problem, as heat_step (right-hand side M (u + dt q), the
 * source term of Eq. RitzGalerkin in the solution's basis); q may be NULL or hold NULLs. */
int bsk_batch_heat_step(bsk_batch* b, void* const* u, const void* const* q, int nsteps,
                        const bsk_cg_opts* opts, bsk_cg_report* reports);

/* Autotuner. The problems of one B-spline degree form a group, whose CG iteration is one
 * persistent launch over (problem, tile, z-chunk) items. For every group it times that launch
 * (`reps` each, CUDA events, finalisers off) for each tile shape -- 64 columns x 16, 24 or 32
 * rows (32 for degrees <= 4 only) -- and each z-chunking (1, 2, 3, 4, 6, 8 chunks per problem),
 * keeps the fastest per group and derives the graph length from the summed iteration time.
 * Overwrites the batch's work vectors. Outputs (may be NULL): graph length, mean ms of one
 * batched iteration (all groups). bsk_batch_groups reports the choices. */
int bsk_batch_autotune(bsk_batch* b, int reps, int* check_every, double* ms);

/* The degree groups of a batch: for group g < min(cap, count) writes its degree, tile rows (16,
 * 24 or 32; tiles are 64 columns wide), z-chunks per problem and autotuned ms per pass (0 if
 * not tuned). Any output array may be NULL. Returns the number of groups (or a negative
 * status). */
int bsk_batch_groups(bsk_batch* b, int cap, int* degree, int* tile_rows, int* nzc, double* ms);

/* Sets the decomposition of the group of `degree` (0: every group) and the graph length directly
 * (e.g. from a cached autotuning result). Returns BSK_EINVAL for a tile shape the degree lacks
 * (tile_rows not 16, 24 or 32; 32 with degree 5) or a degree no problem has. */
int bsk_batch_configure(bsk_batch* b, int degree, int tile_rows, int nzc, int check_every);

/* ---- the learned preconditioner and flexible CG ---------------------------------------------
 * A 3-level convolutional network N maps a normalised residual to an error estimate
 * (16 channels, 3^3 kernels, BF16 weights and activations, FP32 accumulation; the 16 -> 16
 * convolutions run on the 5th-generation tensor cores, tcgen05 MMAs with TMEM accumulators):
 *   a1 = relu(conv_s2(r) + b1); a2 = relu(conv_s2(a1) + b2); a3 = relu(conv_s1(a2) + b3);
 *   a4 = relu(convT_s2(a3) + b4 + a1); z = mask * (convT_s2(a4) + b5 + conv_s1(r; Wf))
 * with stride-2 convolutions halving each axis (ceil) and their transposes restoring it. The
 * paper has no learned component; the network is an addition of this library to the CG stage.
 * Parameters are bsk_net_param_count() FP32 values (layout in net.cu); training runs on the
 * GPU through bsk_net_backward (loss = mean over active voxels of (N(r) - e)^2) and Adam. */
typedef struct bsk_net bsk_net;

int bsk_net_param_count(void);
/* Network for an nx*ny*nz grid (each >= 2); allocates its activations and gradients. */
int bsk_net_create(int nx, int ny, int nz, void* stream, bsk_net** out);
void bsk_net_destroy(bsk_net* net);
/* params: host or device pointer to bsk_net_param_count() floats; resets the Adam state. */
int bsk_net_set_params(bsk_net* net, const float* params);
int bsk_net_get_params(bsk_net* net, float* params);
/* z = N(r); r, z: DEVICE float vectors of the grid; mask: DEVICE uint8 or NULL. */
int bsk_net_forward(bsk_net* net, const float* r, const uint8_t* mask, float* z);
/* Activation of the hidden layers: BSK_ACT_RELU (default) or BSK_ACT_LINEAR (identity, and the
 * biases are ignored and receive no gradient, so the network is a linear map of r: a fixed
 * linear multilevel preconditioner, which flexible CG handles far better than a nonlinear one). */
#define BSK_ACT_RELU 0
#define BSK_ACT_LINEAR 1
int bsk_net_set_activation(bsk_net* net, int act);
/* Zero the accumulated gradients and loss. */
int bsk_net_zero_grad(bsk_net* net);
/* Forward and backward of one sample (r, e): accumulates loss_weight/2 * sum (N(r) - e)^2
 * over active voxels and its parameter gradients (loss_weight = 2 / active voxels gives the
 * mean squared error). */
int bsk_net_backward(bsk_net* net, const float* r, const float* e, const uint8_t* mask, float loss_weight);
/* Forward and backward of one sample for a loss the caller evaluates: dz (DEVICE floats of the
 * grid) is dL/dz, used times scale on active voxels; accumulates the parameter gradients only
 * (the accumulated loss is unchanged). Used for the energy-norm loss
 * (z - e)^T A (z - e), whose gradient 2 A (z - e) needs the operator. */
int bsk_net_backward_grad(bsk_net* net, const float* r, const float* dz, const uint8_t* mask, float scale);
/* Adam step (beta1 0.9, beta2 0.999) with learning rate lr on the gradients times grad_scale. */
int bsk_net_adam(bsk_net* net, float lr, float grad_scale);
/* Accumulated loss (host float) and, if grads is not NULL, the gradients (host floats).
 * bsk_net_read_loss and bsk_net_get_params synchronise the network's stream; they return
 * BSK_ETIMEOUT if a convolution since the network's creation gave up a bounded wait for its
 * loads or MMAs (its outputs were then set to NaN, which flexible CG treats as a failed network
 * and falls back from). */
int bsk_net_read_loss(bsk_net* net, float* loss, float* grads);

/* Not in the paper: the learned preconditioner of this library. Flexible CG (FCG(1), Notay's
 * truncated flexible CG, one previous direction kept A-orthogonal) preconditioned by the network,
 * z = ||r|| N(r / ||r||) / (hx hy hz), as the inner FP32 solver of iterative refinement (handle
 * precision BSK_F32_IR; b, x double). The network must have been created for the handle's grid.
 * An iteration whose network direction is no descent direction (z.r <= 0) uses z = r for that
 * iteration (counted in report->net_rejected); a non-finite network output, or a residual that
 * has not dropped by 2 % within stall_window iterations (default 8), switches the rest of that
 * inner solve to plain CG (report->fallback_iter). The FP64-accurate true residual outside
 * decides convergence, so the network changes the speed, not the answer. net == NULL runs the
 * same iteration without preconditioner (plain CG). The first call allocates the handle's FCG
 * work vectors. */
int fcg_solve(bsk_handle* h, bsk_net* net, const void* b, void* x, const bsk_cg_opts* opts,
              bsk_cg_report* report);

/* The states flexible CG meets, for training the network on them (on-policy pairs). Runs one
 * inner FCG solve of fcg_solve from x = 0 on A d = b / ||b|| (b a DEVICE double vector, handle
 * precision BSK_F32_IR), for `steps` iterations unless it breaks down or stalls, and copies the
 * inner residual r_k = b / ||b|| - A d_k and the iterate d_k (FP32) before each iteration k into
 * r_rec + k n and x_rec + k n (DEVICE float arrays of steps * n elements, n = nx*ny*nz). The
 * solution of A x = b after k iterations is ||b|| d_k, its residual ||b|| r_k. Writes ||b|| to
 * *bnorm (host) and the number of states recorded to *recorded (host; states past a breakdown
 * or stall repeat the last one and are not counted). Uses the handle's FP64 scratch vector. */
int fcg_record(bsk_handle* h, bsk_net* net, const void* b, int steps, float* r_rec, float* x_rec,
               double* bnorm, int* recorded);

/* Kernel timing for roofline measurements. Launches one of the library's kernels `reps` times
 * back to back on the handle's stream, on the handle's own work vectors (which it first zeroes,
 * so any state of a previous solve is lost), and writes the mean device time of one launch in
 * milliseconds (CUDA events on the handle's stream) to *ms. kernel selects:
 *   BSK_KERNEL_OP        y = A x in the CG precision (FP32 for BSK_F32 and BSK_F32_IR)
 *   BSK_KERNEL_CG_FUSED  the fused CG pass: p = r + beta p, x += alpha p_old, q = A p, p.q
 *   BSK_KERNEL_CG_UPDATE the CG residual pass: r -= alpha q, r.r
 *   BSK_KERNEL_RES64     the true residual b - A x in FP64 arithmetic (BSK_F32_IR)
 *   BSK_KERNEL_RES_DF    the same residual in double-float arithmetic (BSK_F32_IR; TMA grids)
 * Returns BSK_EINVAL for an unknown kernel, a kernel the handle does not have, or reps < 1. */
#define BSK_KERNEL_OP 0
#define BSK_KERNEL_CG_FUSED 1
#define BSK_KERNEL_CG_UPDATE 2
#define BSK_KERNEL_RES64 3
#define BSK_KERNEL_RES_DF 4
int bsk_time_kernel(bsk_handle* h, int kernel, int reps, double* ms);

/* Choice of the kernel that runs the single-pass FP32 CG iteration (the CG stage of section 2.5
 * with the operator of Eq. tensForm; bsk_cg_solve, heat_step and the FP32 inner iterations of
 * BSK_F32_IR). Two kernels implement the same iteration on unmasked grids with 16-byte rows
 * and degree <= 4: a warp-specialised pass (BSK_CG_KERNEL_WS: 64 x 32 tiles, one block per SM)
 * and the two-block-per-SM pass used for every other grid (BSK_CG_KERNEL_CLASSIC); neither is
 * the faster on every grid shape. bsk_create chooses with BSK_CG_KERNEL_AUTO, which times
 * three candidates on the handle's own work vectors (zeroing them; about three passes each) and
 * keeps the fastest: the warp-specialised pass with z-chunks of at most 128 planes, the same
 * pass with whole-column items, and the two-block pass. BSK_CG_KERNEL_WS times the first two only.
 * request: BSK_CG_KERNEL_AUTO, BSK_CG_KERNEL_WS, BSK_CG_KERNEL_CLASSIC, or BSK_CG_KERNEL_CURRENT
 * (no change, no timing); *chosen (nullable) receives the kernel now in use (WS or CLASSIC).
 * Call it between solves only, never while the handle's stream is capturing. Returns BSK_EINVAL for an unknown request or for
 * BSK_CG_KERNEL_WS (or _WS_CHUNKED, _WS_COLUMNS) on a handle that cannot use it (masked grid, BSK_F64, degree 5, rows that
 * are not 16-byte multiples); AUTO on such a handle selects CLASSIC without timing. */
#define BSK_CG_KERNEL_AUTO 0
#define BSK_CG_KERNEL_WS 1
#define BSK_CG_KERNEL_CLASSIC 2
#define BSK_CG_KERNEL_CURRENT 3
/* the warp-specialised pass with a fixed item plan, no timing: z-chunks of at most 128 planes, or
 * whole columns */
#define BSK_CG_KERNEL_WS_CHUNKED 4
#define BSK_CG_KERNEL_WS_COLUMNS 5
int bsk_select_cg_kernel(bsk_handle* h, int request, int* chosen);

/* The CG kernel in use (BSK_CG_KERNEL_WS or _CLASSIC) and, for the warp-specialised pass, the
 * most planes per z-chunk its items take (the whole column when that was faster). Either output
 * may be NULL. */
int bsk_cg_kernel_config(bsk_handle* h, int* kernel, int* zchunk_planes);

/* Allocation-free residual: r = b - A x (A as for op_apply), with *rr = r.r and *bb = b.b
 * reduced in FP64. The paper has no counterpart for this interface: it serves callers that
 * cannot allocate device memory -- for example a solver plugin inside a host application that
 * owns the device memory budget and hands in pre-allocated buffers -- and therefore cannot
 * create a handle.
 * It needs no handle and allocates nothing: its scratch (an FP64 scalar block and the partial
 * sums of the two reductions, about 256 KB) is a file-scope static device array that every GPU
 * loading this library holds until the process exits. prob describes the grid as for
 * bsk_create (prob->mask, if set, is read in place); precision is BSK_F64 (double vectors) or
 * BSK_F32 (float vectors; reductions still FP64); x, b, r are DEVICE vectors of nx*ny*nz
 * elements owned by the caller, r must not overlap x or b; stream is a cudaStream_t.
 * The first call on a device looks up the scratch's device address with that device current
 * (and the first call per precision and degree sets up that operator kernel); make that first
 * call before any stream capture. Every call reads its two norms back to the host and
 * synchronises `stream`; a call made while `stream` is capturing returns BSK_EINVAL without
 * touching the capture.
 * Every call shares the one scratch array and clears what must start at zero itself; calls
 * that overlap on the GPU (other streams, other threads) race on it and must be serialised by
 * the caller.
 * Returns BSK_EINVAL (with a message in bsk_last_error) for a grid with
 * ceil(nx/32) * ceil(ny/16) > 16384 (about 8.4 M nodes per x-y plane; nz is not limited), for
 * bad arguments, or for precision BSK_F32_IR. */
int residual_noalloc(const bsk_problem* prob, int precision, const void* x, const void* b, void* r,
                     double* rr, double* bb, void* stream);

/* ---- z-slab split of one grid across devices (section 3 distributes the unknowns of one
 * problem over several GPUs; here each device holds a contiguous range of z-planes) ----
 *
 * A slab handle is an ordinary handle created (bsk_create) for the LOCAL grid nx x ny x nz of
 * one slab (precision BSK_F64 or BSK_F32, no mask, odd reflection at the faces, constant
 * coefficients), then told where the slab sits with bsk_set_slab. The slab calls below then
 * treat its nz planes as planes z_off .. z_off + nz - 1 of a grid of nz_glob planes: the
 * operator of Eq. tensForm couples a plane to the n planes on each side, so inputs of the
 * operator carry n HALO planes on each side (nz + 2n planes, plane i of the array being global
 * plane z_off - n + i), and odd reflection applies at the global faces z = 0 and z = nz_glob - 1
 * only (halo planes beyond a global face are never read). Halo planes are the caller's to fill
 * from the neighbouring slabs (NCCL send/recv, peer copies, host copies).
 * The other calls (op_apply, bsk_cg_solve, ...) keep treating the handle as a whole grid of nz
 * planes. Vectors are DEVICE arrays of the handle's element type owned by the caller. */

/* Places the handle's grid as planes z_off .. z_off + nz - 1 of a grid of nz_glob planes.
 * Returns BSK_EINVAL for z_off < 0, z_off + nz > nz_glob, or a handle that is not of the kind
 * described above. */
int bsk_set_slab(bsk_handle* h, int z_off, int nz_glob);

/* y = A x on the slab's planes (A of Eq. tensForm, as for op_apply), x_halo holding nz + 2n
 * planes (n halo planes below and above the local ones), y the nz local planes. x_halo and y
 * must not overlap. Asynchronous on the handle's stream. */
int bsk_slab_apply(bsk_handle* h, const void* x_halo, void* y);

/* Scalars of a slab CG solve: a DEVICE array of BSK_SLAB_SCALARS doubles owned by the caller,
 * on which the all-reduces act in place. Between the passes below the caller sums, over all
 * slabs of the grid, the entries the previous pass left as local partial sums:
 *   after bsk_slab_cg_begin:  RR_NEW and BB (2 doubles from BSK_SLAB_RR_NEW)
 *   after bsk_slab_cg_matvec: PQ (1 double at BSK_SLAB_PQ)
 *   after bsk_slab_cg_update: RR_NEW (1 double at BSK_SLAB_RR_NEW)
 * DONE becomes 1 when the solve has ended (on every slab alike, the scalars being global), with
 * STATUS 0 (converged: r.r <= tol^2 b.b), 1 (max_iter iterations) or -5 (breakdown: p.Ap <= 0 or
 * a non-finite norm); ITER counts the iterations and RR holds the last global r.r. Passes
 * launched after DONE change neither x nor r, so a caller may queue several iterations between
 * reads of DONE. */
#define BSK_SLAB_PQ 0
#define BSK_SLAB_RR_NEW 1
#define BSK_SLAB_BB 2
#define BSK_SLAB_RR 3
#define BSK_SLAB_TOL2 4
#define BSK_SLAB_MAX_ITER 5
#define BSK_SLAB_ITER 6
#define BSK_SLAB_DONE 7
#define BSK_SLAB_STATUS 8
#define BSK_SLAB_SCALARS 16

/* Starts CG (section 2.5) on a slab: r = b - ax, p = r (local planes of p_halo, which holds
 * nz + 2n planes), with ax = A x0 computed by the caller (bsk_slab_apply on the halo-extended
 * x0, or zeros for x0 = 0); resets s for tolerance tol (relative, ||r|| <= tol ||b||) and
 * max_iter; leaves local r.r and b.b in s. After the all-reduce, call
 * bsk_slab_cg_direction(first = 1). r, b, ax are nz-plane vectors. */
int bsk_slab_cg_begin(bsk_handle* h, const void* b, const void* ax, void* r, void* p_halo, double* s,
                      double tol, int max_iter);

/* q = A p (p_halo with filled halo planes) and local p.q into s. */
int bsk_slab_cg_matvec(bsk_handle* h, const void* p_halo, void* q, double* s);

/* alpha = RR / PQ; x += alpha p, r -= alpha q on the local planes; local r.r into s. */
int bsk_slab_cg_update(bsk_handle* h, void* x, void* r, const void* p_halo, const void* q, double* s);

/* p = r + beta p on the local planes of p_halo, beta = RR_NEW / RR (0 when first is non-zero),
 * then the convergence test; the halo planes of p are to be exchanged before the next matvec. */
int bsk_slab_cg_direction(bsk_handle* h, const void* r, void* p_halo, double* s, int first);

/* out = 1 / diag A per node (the Jacobi scaling of bsk_set_preconditioner: for constant
 * coefficients the diagonal of the separable operator of Eq. tensForm including the mirror images
 * near the faces, with the boundary term for Robin handles; probed for variable coefficients;
 * zero on inactive nodes of a mask). out is a DEVICE vector of nx*ny*nz elements of the handle's
 * element type (BSK_F64 or BSK_F32 handles). Returns BSK_EINVAL when the handle has no Jacobi
 * preconditioner set. Asynchronous on the handle's stream. */
int bsk_inverse_diagonal(bsk_handle* h, void* out);

/* heat_step on HOST buffers: copies u (and q, if not NULL) from the host to device vectors the
 * handle keeps for this purpose (allocated by the first call), runs heat_step there, and copies
 * the new u back into u_host, all on the handle's stream; returns after the copy back. u_host and
 * q_host are HOST arrays of nx*ny*nz elements of the handle's element type; pinned memory
 * (cudaHostAlloc, or torch's pin_memory) lets the copies run at the link's speed, pageable
 * memory works but is staged by the driver. report (may be NULL) is heat_step's, with h2d_ms and
 * d2h_ms the device times of the copies and elapsed_ms the whole call. */
int heat_step_host(bsk_handle* h, void* u_host, const void* q_host, int nsteps, const bsk_cg_opts* opts,
                   bsk_cg_report* report);

/* Text of the last error raised on the calling thread ("" if none). */
const char* bsk_last_error(void);

/* Human-readable name of a status code. */
const char* bsk_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* BSK_H */
