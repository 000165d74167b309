/*
 * bsk_oracle.c -- plain FP64 CPU oracle for the tensor B-spline heat-equation operator.
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library. The CUDA product path never links, imports or calls it, and
 * it shares no code, header, table or helper with that path.
 *
 * Everything is double precision, round-to-nearest, with no blocking or fusion beyond what the
 * paper's definitions state. Passages followed (paper arXiv:1904.03057):
 *   - B-spline definition and identities: Table tblBsplines (section 2.3): convolution,
 *     derivative and scalar-product rows.
 *   - Tensor-product basis: section 2.3, the multivariate B-spline definition.
 *   - Galerkin system: Eq. RitzGalerkin (section 2.3) and Eq. tensForm (section 2.4) with
 *     constant coefficients, D = dt and mu_a = 1 (one implicit Euler step of the heat equation).
 *   - Separable shift-invariant kernels and the filtering algorithm: section 2.4 and
 *     Fig. FiltAlg (four chains of three 1-D convolutions summed into p).
 *   - Variable coefficients: Eq. RitzGalerkin and Eq. tensForm with D(x) and mu_a(x) expanded
 *     in B-splines (section 2.3), the on-the-fly strategy of section 2.4 written as the plain
 *     double sum over solution and coefficient B-splines with 1-D triple-product factors.
 *   - Boundary penalty (Robin) problems on the box: the boundary integral of Eq. RitzGalerkin
 *     over the untruncated basis; the Jacobi-preconditioned CG and the coarse-grid
 *     initialisation of the large run of section 3.
 *   - Conjugate gradient: section 2.5 (Fig. figGenTenSolv, stage 3).
 *   - Indirect B-spline transform (evaluation): section 2.3, Fig. figBspnSignProc.
 *   - L2 norm: Appendix I.
 *
 * Readings where the paper is silent (zero Dirichlet faces by odd reflection, node masks for
 * curved domains, h = 1/(N+1)) are the ones listed in the design notes of the repository.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;        /* unknowns per axis; array layout [nz][ny][nx], x fastest     */
    int n;                 /* B-spline degree                                            */
    double hx, hy, hz;     /* grid steps                                                 */
    double dt;             /* weight of the stiffness term (implicit Euler time step)    */
    const uint8_t* mask;   /* [nz][ny][nx] node mask, 1 = active; NULL = whole box       */
} orc_problem;

/* ------------------------------------------------------------------------------------------ */
/* 1-D B-splines                                                                               */
/* ------------------------------------------------------------------------------------------ */

/* Centred B-spline beta^n(x). beta^0 is the unit box on [-1/2, 1/2); beta^n is the (n+1)-fold
 * self-convolution of beta^0 (Table tblBsplines, convolution row). The two-term recurrence
 * used here follows from that convolution definition (de Boor's recurrence for uniform knots,
 * re-centred). */
double orc_bspline(int n, double x)
{
    if (n == 0) return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    double half = 0.5 * (double)(n + 1);
    if (x <= -half || x >= half) return 0.0;
    return ((half + x) * orc_bspline(n - 1, x + 0.5) + (half - x) * orc_bspline(n - 1, x - 0.5)) /
           (double)n;
}

/* Derivative: beta^n'(x) = beta^{n-1}(x + 1/2) - beta^{n-1}(x - 1/2) (Table tblBsplines). */
double orc_bspline_deriv(int n, double x)
{
    if (n < 1) return 0.0;
    return orc_bspline(n - 1, x + 0.5) - orc_bspline(n - 1, x - 0.5);
}

/* Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the Legendre polynomial). */
static void gauss_legendre(int m, double* t, double* w)
{
    for (int i = 0; i < m; i++) {
        double x = cos(M_PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p1 = x; p0 = 1.0; }
            dp = m * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p1 = x; p0 = 1.0; }
            dp = m * (x * p1 - p0) / (x * x - 1.0);
        }
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

int orc_gauss_legendre(int m, double* t, double* w)
{
    if (m < 1 || m > 64) return -1;
    gauss_legendre(m, t, w);
    return 0;
}

/* 1-D Galerkin kernels on a unit grid, by quadrature of the defining integrals:
 *   mass      m_j = integral beta^n(x) beta^n(x - j) dx
 *   stiffness k_j = integral beta^n'(x) beta^n'(x - j) dx,     j = -n..n,
 * stored at index j + n. Both integrands are piecewise polynomials of degree <= 2n whose
 * breakpoints are the knots of beta^n, so n+1 Gauss points per unit knot interval integrate
 * them exactly. (The paper states the closed forms through the scalar-product identity of
 * Table tblBsplines; this routine computes the integrals themselves.) */
int orc_kernels_1d(int n, double* m, double* k)
{
    if (n < 1 || n > 7) return -1;
    double t[16], w[16];
    int q = n + 1;
    gauss_legendre(q, t, w);
    double half = 0.5 * (double)(n + 1);
    for (int j = 0; j <= n; j++) {
        double sm = 0.0, sk = 0.0;
        for (int iv = 0; iv <= n; iv++) {
            double a = -half + iv, b = a + 1.0;
            for (int g = 0; g < q; g++) {
                double x = 0.5 * (a + b) + 0.5 * (b - a) * t[g];
                double wt = 0.5 * (b - a) * w[g];
                sm += wt * orc_bspline(n, x) * orc_bspline(n, x - j);
                sk += wt * orc_bspline_deriv(n, x) * orc_bspline_deriv(n, x - j);
            }
        }
        m[n + j] = m[n - j] = sm;
        k[n + j] = k[n - j] = sk;
    }
    return 0;
}

/* Per-axis kernels for grid step h: M = h * m, K = k / h (Galerkin integrals of the
 * scaled basis beta^n(x/h - i)). */
int orc_bspline_kernels(int n, double h, double* M, double* K)
{
    if (!(h > 0.0)) return -1;
    if (orc_kernels_1d(n, M, K) != 0) return -1;
    for (int j = 0; j < 2 * n + 1; j++) {
        M[j] *= h;
        K[j] /= h;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Ghost extension: zero Dirichlet faces by odd reflection, node mask                          */
/* ------------------------------------------------------------------------------------------ */

/* Reflected index of array position a (0-based) on an axis of N unknowns. The box faces sit at
 * positions -1 and N, where the coefficient is zero; beyond them the coefficient is minus its
 * mirror image. Returns 0 for a zero ghost, else +1/-1 and the source index in *src. */
static int reflect(int a, int N, int* src)
{
    if (a >= 0 && a < N) { *src = a; return 1; }
    int r = (a < 0) ? (-2 - a) : (2 * N - a);
    if (r < 0 || r >= N) return 0; /* the face itself (or beyond one reflection: never used) */
    *src = r;
    return -1;
}

/* Deliberate-mistake switch for the test-suite's planted-error checks: 0 = correct odd
 * reflection (default), 1 = zero ghosts, 2 = even reflection, 3 = zero ghosts for the
 * coefficient fields of the variable-coefficient operator, 4 = the far face left out of the
 * Robin boundary term. Tests set it, check that a pin fails, and reset it. */
static int g_plant = 0;
void orc_set_plant(int mode) { g_plant = mode; }

/* E = masked, odd-reflected copy of x on [-n, N+n) per axis; E dims (nz+2n)(ny+2n)(nx+2n).
 * With absmode set, E holds |x| at interior points and at ghosts (used for error scales). */
static double* extend_mode(const orc_problem* p, const double* x, int absmode)
{
    int n = p->n;
    int ex = p->nx + 2 * n, ey = p->ny + 2 * n, ez = p->nz + 2 * n;
    double* E = (double*)malloc(sizeof(double) * (size_t)ex * ey * ez);
    if (!E) return NULL;
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < ez; kz++) {
        for (int ky = 0; ky < ey; ky++) {
            for (int kx = 0; kx < ex; kx++) {
                int sz, sy, sx;
                int s = reflect(kz - n, p->nz, &sz);
                s *= (s ? reflect(ky - n, p->ny, &sy) : 0);
                s *= (s ? reflect(kx - n, p->nx, &sx) : 0);
                double v = 0.0;
                if (s) {
                    size_t src = ((size_t)sz * p->ny + sy) * p->nx + sx;
                    if (g_plant == 1 && s < 0) s = 0;
                    if (g_plant == 2 && s < 0) s = 1;
                    v = (p->mask && !p->mask[src]) ? 0.0 : s * x[src];
                    if (absmode) v = fabs(v);
                }
                E[((size_t)kz * ey + ky) * ex + kx] = v;
            }
        }
    }
    return E;
}

static double* extend(const orc_problem* p, const double* x) { return extend_mode(p, x, 0); }

static int problem_ok(const orc_problem* p)
{
    if (!p || p->n < 1 || p->n > 7) return 0;
    if (p->nx < p->n || p->ny < p->n || p->nz < p->n) return 0;
    if (!(p->hx > 0 && p->hy > 0 && p->hz > 0)) return 0;
    return 1;
}

/* Kernel block layout used by the operator routines: kern = [Mx | Kx | My | Ky | Mz | Kz],
 * each of length 2n+1. Passing the kernels explicitly lets a test feed deliberately wrong
 * kernels and check that the independent pins catch them. */
int orc_problem_kernels(const orc_problem* p, double* kern)
{
    if (!problem_ok(p)) return -1;
    int L = 2 * p->n + 1;
    if (orc_bspline_kernels(p->n, p->hx, kern + 0 * L, kern + 1 * L)) return -1;
    if (orc_bspline_kernels(p->n, p->hy, kern + 2 * L, kern + 3 * L)) return -1;
    if (orc_bspline_kernels(p->n, p->hz, kern + 4 * L, kern + 5 * L)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Operator, definition form: direct (2n+1)^3 stencil                                         */
/* ------------------------------------------------------------------------------------------ */

/* y = mask o [ (Mz x My x Mx) + dt (Kz x My x Mx + Mz x Ky x Mx + Mz x My x Kx) ] (mask o x),
 * with odd-reflected ghosts: the constant-coefficient case of Eq. tensForm, written as one
 * shift-invariant 3-D stencil whose weights are the tensor products of the 1-D kernels
 * (section 2.4, separability of the kernels). Summation runs over the full 3-D stencil. */
int orc_op_stencil(const orc_problem* p, const double* kern, const double* x, double* y)
{
    if (!problem_ok(p)) return -1;
    int n = p->n, L = 2 * n + 1;
    const double *Mx = kern, *Kx = kern + L, *My = kern + 2 * L, *Ky = kern + 3 * L;
    const double *Mz = kern + 4 * L, *Kz = kern + 5 * L;
    double* W = (double*)malloc(sizeof(double) * L * L * L);
    if (!W) return -3;
    for (int c = 0; c < L; c++)
        for (int b = 0; b < L; b++)
            for (int a = 0; a < L; a++)
                W[(c * L + b) * L + a] = Mz[c] * My[b] * Mx[a] +
                                         p->dt * (Kz[c] * My[b] * Mx[a] + Mz[c] * Ky[b] * Mx[a] +
                                                  Mz[c] * My[b] * Kx[a]);
    double* E = extend(p, x);
    if (!E) { free(W); return -3; }
    int ex = p->nx + 2 * n, ey = p->ny + 2 * n;
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; iz++) {
        for (int iy = 0; iy < p->ny; iy++) {
            for (int ix = 0; ix < p->nx; ix++) {
                size_t o = ((size_t)iz * p->ny + iy) * p->nx + ix;
                if (p->mask && !p->mask[o]) { y[o] = 0.0; continue; }
                double s = 0.0;
                for (int c = 0; c < L; c++)
                    for (int b = 0; b < L; b++)
                        for (int a = 0; a < L; a++)
                            s += W[(c * L + b) * L + a] *
                                 E[((size_t)(iz + c) * ey + (iy + b)) * ex + (ix + a)];
                y[o] = s;
            }
        }
    }
    free(E);
    free(W);
    return 0;
}

/* The same definition evaluated at selected points only, for parity checks at sizes where a
 * full oracle pass is too slow: y at each flat index pts[i] (array order), with x read as float
 * (x_is_f32 != 0) or double. Ghost values follow the same odd-reflection and mask rules. */
int orc_op_points(const orc_problem* p, const double* kern, const void* x, int x_is_f32,
                  long long npts, const long long* pts, double* out)
{
    if (!problem_ok(p)) return -1;
    int n = p->n, L = 2 * n + 1;
    const double *Mx = kern, *Kx = kern + L, *My = kern + 2 * L, *Ky = kern + 3 * L;
    const double *Mz = kern + 4 * L, *Kz = kern + 5 * L;
    double* W = (double*)malloc(sizeof(double) * L * L * L);
    if (!W) return -3;
    for (int c = 0; c < L; c++)
        for (int b = 0; b < L; b++)
            for (int a = 0; a < L; a++)
                W[(c * L + b) * L + a] = Mz[c] * My[b] * Mx[a] +
                                         p->dt * (Kz[c] * My[b] * Mx[a] + Mz[c] * Ky[b] * Mx[a] +
                                                  Mz[c] * My[b] * Kx[a]);
    const float* xf = (const float*)x;
    const double* xd = (const double*)x;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < npts; t++) {
        long long I = pts[t];
        int ix = (int)(I % p->nx), iy = (int)((I / p->nx) % p->ny);
        int iz = (int)(I / ((long long)p->nx * p->ny));
        if (p->mask && !p->mask[I]) { out[t] = 0.0; continue; }
        double s = 0.0;
        for (int c = 0; c < L; c++) {
            int sz, sgn_z = reflect(iz + c - n, p->nz, &sz);
            if (!sgn_z) continue;
            for (int b = 0; b < L; b++) {
                int sy, sgn_y = reflect(iy + b - n, p->ny, &sy);
                if (!sgn_y) continue;
                for (int a = 0; a < L; a++) {
                    int sx, sgn_x = reflect(ix + a - n, p->nx, &sx);
                    if (!sgn_x) continue;
                    size_t src = ((size_t)sz * p->ny + sy) * p->nx + sx;
                    if (p->mask && !p->mask[src]) continue;
                    double v = x_is_f32 ? (double)xf[src] : xd[src];
                    s += W[(c * L + b) * L + a] * (sgn_z * sgn_y * sgn_x) * v;
                }
            }
        }
        out[t] = s;
    }
    free(W);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Operator, the paper's filtering algorithm: separable 1-D convolution chains                 */
/* ------------------------------------------------------------------------------------------ */

/* "Valid" correlation of in (dims d[0]=x, d[1]=y, d[2]=z) with a symmetric (2n+1)-tap kernel
 * along one axis; the output is 2n shorter along that axis. */
static void conv_axis(const double* in, const int* d, int axis, const double* t, int n, double* out)
{
    int o[3] = {d[0], d[1], d[2]};
    o[axis] -= 2 * n;
    size_t stride = axis == 0 ? 1 : axis == 1 ? (size_t)d[0] : (size_t)d[0] * d[1];
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < o[2]; kz++)
        for (int ky = 0; ky < o[1]; ky++)
            for (int kx = 0; kx < o[0]; kx++) {
                size_t base = ((size_t)kz * d[1] + ky) * d[0] + kx;
                double s = 0.0;
                for (int j = 0; j < 2 * n + 1; j++) s += t[j] * in[base + j * stride];
                out[((size_t)kz * o[1] + ky) * o[0] + kx] = s;
            }
}

/* p = dt (d * w_x f_y f_z) + dt (d * f_x w_y f_z) + dt (d * f_x f_y w_z) + (m * f_x f_y f_z)
 * with d == 1, m == 1 (constant coefficients), w = stiffness and f = mass kernels: the four
 * chains of Fig. FiltAlg, each a sequence of three 1-D convolutions along axes 1, 2, 3
 * (x, y, z here), applied to the ghost-extended coefficients and summed. With mass_only set,
 * only the last chain runs (the mass operator used for right-hand sides). */
static int op_separable(const orc_problem* p, const double* kern, const double* x, double* y,
                        int mass_only, int absmode)
{
    if (!problem_ok(p)) return -1;
    int n = p->n, L = 2 * n + 1;
    const double* Mk[3] = {kern, kern + 2 * L, kern + 4 * L};
    const double* Kk[3] = {kern + L, kern + 3 * L, kern + 5 * L};
    double* E = extend_mode(p, x, absmode);
    if (!E) return -3;
    int d0[3] = {p->nx + 2 * n, p->ny + 2 * n, p->nz + 2 * n};
    size_t nout = (size_t)p->nx * p->ny * p->nz;
    int d1[3] = {p->nx, d0[1], d0[2]};
    int d2[3] = {p->nx, p->ny, d0[2]};
    double* t1 = (double*)malloc(sizeof(double) * (size_t)d1[0] * d1[1] * d1[2]);
    double* t2 = (double*)malloc(sizeof(double) * (size_t)d2[0] * d2[1] * d2[2]);
    double* t3 = (double*)malloc(sizeof(double) * nout);
    if (!t1 || !t2 || !t3) { free(E); free(t1); free(t2); free(t3); return -3; }
    memset(y, 0, sizeof(double) * nout);
    for (int chain = 0; chain < 4; chain++) {
        if (mass_only && chain < 3) continue;
        /* chain c < 3 puts the stiffness kernel on axis c; chain 3 is mass on every axis */
        const double* tx = chain == 0 ? Kk[0] : Mk[0];
        const double* ty = chain == 1 ? Kk[1] : Mk[1];
        const double* tz = chain == 2 ? Kk[2] : Mk[2];
        double wgt = chain < 3 ? p->dt : 1.0;
        conv_axis(E, d0, 0, tx, n, t1);
        conv_axis(t1, d1, 1, ty, n, t2);
        conv_axis(t2, d2, 2, tz, n, t3);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)nout; i++) y[i] += wgt * t3[i];
    }
    if (p->mask) {
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)nout; i++)
            if (!p->mask[i]) y[i] = 0.0;
    }
    free(E);
    free(t1);
    free(t2);
    free(t3);
    return 0;
}

int orc_op_separable(const orc_problem* p, const double* kern, const double* x, double* y)
{
    return op_separable(p, kern, x, y, 0, 0);
}

int orc_mass(const orc_problem* p, const double* kern, const double* x, double* y)
{
    return op_separable(p, kern, x, y, 1, 0);
}

/* (|A| |x|)_i: every kernel tap and every (ghost-extended) coefficient replaced by its absolute
 * value. This bounds the magnitude of the terms summed into (A x)_i and is the scale against
 * which operator rounding errors are measured (the stiffness kernel sums to zero, so (A x)_i
 * itself can be far smaller than its terms). */
int orc_abs_op(const orc_problem* p, const double* kern, const double* x, double* y)
{
    if (!problem_ok(p)) return -1;
    int L = 2 * p->n + 1;
    double* ak = (double*)malloc(sizeof(double) * 6 * L);
    if (!ak) return -3;
    for (int i = 0; i < 6 * L; i++) ak[i] = fabs(kern[i]);
    orc_problem q = *p;
    q.dt = fabs(p->dt);
    int rc = op_separable(&q, ak, x, y, 0, 1);
    free(ak);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Brute-force Galerkin matrix on tiny grids                                                   */
/* ------------------------------------------------------------------------------------------ */

/* 1-D basis with zero Dirichlet faces at 0 and (N+1)h: the tensor B-spline centred at i h,
 * minus its mirror images in both faces (odd, 2(N+1)h-periodic extension), i = 1..N. */
static double psi_1d(int n, int N, double h, int i, double x, int deriv)
{
    double s = 0.0, u = x / h;
    for (int k = -1; k <= 1; k++) {
        double shift = 2.0 * k * (N + 1);
        if (deriv) {
            s += orc_bspline_deriv(n, u - i - shift) - orc_bspline_deriv(n, u + i - shift);
        } else {
            s += orc_bspline(n, u - i - shift) - orc_bspline(n, u + i - shift);
        }
    }
    return deriv ? s / h : s;
}

/* Quadrature rule on [0, (N+1)h]: sub-intervals of length h/2 (they contain every knot of
 * both even and odd degree), n+1 Gauss points each. Returns the number of points. */
static int axis_rule(int n, int N, double h, double* xs, double* ws)
{
    double t[16], w[16];
    int q = n + 1, cnt = 0;
    gauss_legendre(q, t, w);
    for (int c = 0; c < 2 * (N + 1); c++) {
        double a = 0.5 * h * c, b = a + 0.5 * h;
        for (int g = 0; g < q; g++) {
            xs[cnt] = 0.5 * (a + b) + 0.5 * (b - a) * t[g];
            ws[cnt] = 0.5 * (b - a) * w[g];
            cnt++;
        }
    }
    return cnt;
}

/* A_ij = integral over [0,1]^3 of ( psi_i psi_j + dt grad psi_i . grad psi_j ) for active i, j
 * (Eq. RitzGalerkin with D = dt, mu_a = 1, no boundary term: the basis vanishes on the faces),
 * assembled by Gauss quadrature from point values of the basis. The active nodes are
 * numbered in array order; A is na x na, row-major. With full3d set the integral is summed
 * over the 3-D tensor quadrature grid point by point; otherwise it is factorised by Fubini
 * into 1-D Gram matrices (same integral, fewer operations). */
int orc_bruteforce_matrix(const orc_problem* p, int full3d, double* A, int* na_out)
{
    if (!problem_ok(p)) return -1;
    int n = p->n, N[3] = {p->nx, p->ny, p->nz};
    double h[3] = {p->hx, p->hy, p->hz};
    size_t ntot = (size_t)N[0] * N[1] * N[2];
    int* act = (int*)malloc(sizeof(int) * ntot);
    int na = 0;
    for (size_t i = 0; i < ntot; i++) act[i] = (!p->mask || p->mask[i]) ? na++ : -1;
    *na_out = na;
    if (!A) { free(act); return 0; }
    /* 1-D tables: value and derivative of each basis function at each quadrature point */
    double* xs[3]; double* ws[3]; double* B[3]; double* D[3]; int nq[3];
    for (int d = 0; d < 3; d++) {
        int maxq = 2 * (N[d] + 1) * (n + 1);
        xs[d] = (double*)malloc(sizeof(double) * maxq);
        ws[d] = (double*)malloc(sizeof(double) * maxq);
        nq[d] = axis_rule(n, N[d], h[d], xs[d], ws[d]);
        B[d] = (double*)malloc(sizeof(double) * (size_t)N[d] * nq[d]);
        D[d] = (double*)malloc(sizeof(double) * (size_t)N[d] * nq[d]);
        for (int i = 0; i < N[d]; i++)
            for (int q = 0; q < nq[d]; q++) {
                B[d][(size_t)i * nq[d] + q] = psi_1d(n, N[d], h[d], i + 1, xs[d][q], 0);
                D[d][(size_t)i * nq[d] + q] = psi_1d(n, N[d], h[d], i + 1, xs[d][q], 1);
            }
    }
    memset(A, 0, sizeof(double) * (size_t)na * na);
    double* GM[3]; double* GK[3];
    for (int d = 0; d < 3; d++) {
        GM[d] = (double*)calloc((size_t)N[d] * N[d], sizeof(double));
        GK[d] = (double*)calloc((size_t)N[d] * N[d], sizeof(double));
        for (int i = 0; i < N[d]; i++)
            for (int j = 0; j < N[d]; j++) {
                double sm = 0, sk = 0;
                for (int q = 0; q < nq[d]; q++) {
                    sm += ws[d][q] * B[d][(size_t)i * nq[d] + q] * B[d][(size_t)j * nq[d] + q];
                    sk += ws[d][q] * D[d][(size_t)i * nq[d] + q] * D[d][(size_t)j * nq[d] + q];
                }
                GM[d][i * N[d] + j] = sm;
                GK[d][i * N[d] + j] = sk;
            }
    }
#pragma omp parallel for schedule(dynamic)
    for (long long I = 0; I < (long long)ntot; I++) {
        if (act[I] < 0) continue;
        int ix = (int)(I % N[0]), iy = (int)((I / N[0]) % N[1]), iz = (int)(I / ((size_t)N[0] * N[1]));
        for (size_t J = 0; J < ntot; J++) {
            if (act[J] < 0) continue;
            int jx = (int)(J % N[0]), jy = (int)((J / N[0]) % N[1]), jz = (int)(J / ((size_t)N[0] * N[1]));
            double v;
            if (full3d) {
                v = 0.0;
                for (int qz = 0; qz < nq[2]; qz++) {
                    double bz_i = B[2][(size_t)iz * nq[2] + qz], bz_j = B[2][(size_t)jz * nq[2] + qz];
                    double dz_i = D[2][(size_t)iz * nq[2] + qz], dz_j = D[2][(size_t)jz * nq[2] + qz];
                    if (bz_i == 0 && bz_j == 0 && dz_i == 0 && dz_j == 0) continue;
                    for (int qy = 0; qy < nq[1]; qy++) {
                        double by_i = B[1][(size_t)iy * nq[1] + qy], by_j = B[1][(size_t)jy * nq[1] + qy];
                        double dy_i = D[1][(size_t)iy * nq[1] + qy], dy_j = D[1][(size_t)jy * nq[1] + qy];
                        for (int qx = 0; qx < nq[0]; qx++) {
                            double bx_i = B[0][(size_t)ix * nq[0] + qx], bx_j = B[0][(size_t)jx * nq[0] + qx];
                            double dx_i = D[0][(size_t)ix * nq[0] + qx], dx_j = D[0][(size_t)jx * nq[0] + qx];
                            double w = ws[2][qz] * ws[1][qy] * ws[0][qx];
                            double pi = bz_i * by_i * bx_i, pj = bz_j * by_j * bx_j;
                            double g = (dz_i * by_i * bx_i) * (dz_j * by_j * bx_j) +
                                       (bz_i * dy_i * bx_i) * (bz_j * dy_j * bx_j) +
                                       (bz_i * by_i * dx_i) * (bz_j * by_j * dx_j);
                            v += w * (pi * pj + p->dt * g);
                        }
                    }
                }
            } else {
                double mx = GM[0][ix * N[0] + jx], my = GM[1][iy * N[1] + jy], mz = GM[2][iz * N[2] + jz];
                double kx = GK[0][ix * N[0] + jx], ky = GK[1][iy * N[1] + jy], kz = GK[2][iz * N[2] + jz];
                v = mz * my * mx + p->dt * (kz * my * mx + mz * ky * mx + mz * my * kx);
            }
            A[(size_t)act[I] * na + act[J]] = v;
        }
    }
    for (int d = 0; d < 3; d++) { free(xs[d]); free(ws[d]); free(B[d]); free(D[d]); free(GM[d]); free(GK[d]); }
    free(act);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Vectors and conjugate gradient                                                              */
/* ------------------------------------------------------------------------------------------ */

/* Deterministic dot product: fixed chunks of 4096 summed in a fixed order, whatever the
 * number of threads. */
static double dot(const double* a, const double* b, size_t len)
{
    size_t nchunk = (len + 4095) / 4096;
    double* part = (double*)malloc(sizeof(double) * (nchunk ? nchunk : 1));
#pragma omp parallel for schedule(static)
    for (long long c = 0; c < (long long)nchunk; c++) {
        size_t lo = (size_t)c * 4096, hi = lo + 4096 < len ? lo + 4096 : len;
        double s = 0.0;
        for (size_t i = lo; i < hi; i++) s += a[i] * b[i];
        part[c] = s;
    }
    double s = 0.0;
    for (size_t c = 0; c < nchunk; c++) s += part[c];
    free(part);
    return s;
}

double orc_dot(const double* a, const double* b, long long len) { return dot(a, b, (size_t)len); }

/* Textbook conjugate gradient (Hestenes-Stiefel) for A x = b, A from orc_op_separable
 * (section 2.5: the iterative solver of F(c) = t). Stops when the recursively updated residual
 * satisfies ||r|| <= tol ||b||. On return *iters holds the iteration count and *relres the
 * true relative residual ||b - A x|| / ||b|| recomputed from x. Entries of b and x at inactive
 * nodes are treated as zero (x is zeroed there). Returns 0 if converged, 1 if max_iter was
 * reached, -5 on breakdown (p.Ap <= 0 or NaN). */
int orc_cg(const orc_problem* p, const double* kern, const double* b, double* x, double tol,
           int max_iter, int* iters, double* relres)
{
    if (!problem_ok(p)) return -1;
    size_t len = (size_t)p->nx * p->ny * p->nz;
    double* r = (double*)malloc(sizeof(double) * len);
    double* pv = (double*)malloc(sizeof(double) * len);
    double* q = (double*)malloc(sizeof(double) * len);
    if (!r || !pv || !q) { free(r); free(pv); free(q); return -3; }
    int status = 1, it = 0;
    /* the system lives on the active nodes: inactive entries of b and x are treated as zero */
    double* bm = (double*)malloc(sizeof(double) * len);
    if (!bm) { free(r); free(pv); free(q); return -3; }
    for (size_t i = 0; i < len; i++) {
        int act = !p->mask || p->mask[i];
        bm[i] = act ? b[i] : 0.0;
        if (!act) x[i] = 0.0;
    }
    b = bm;
    double bb = dot(b, b, len);
    orc_op_separable(p, kern, x, q);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)len; i++) { r[i] = b[i] - q[i]; pv[i] = r[i]; }
    double rr = dot(r, r, len);
    if (bb == 0.0) {
        memset(x, 0, sizeof(double) * len);
        status = 0;
    } else if (sqrt(rr) <= tol * sqrt(bb)) {
        status = 0;
    } else {
        for (it = 1; it <= max_iter; it++) {
            orc_op_separable(p, kern, pv, q);
            double pq = dot(pv, q, len);
            if (!(pq > 0.0)) { status = -5; break; }
            double alpha = rr / pq;
#pragma omp parallel for schedule(static)
            for (long long i = 0; i < (long long)len; i++) {
                x[i] += alpha * pv[i];
                r[i] -= alpha * q[i];
            }
            double rr_new = dot(r, r, len);
            if (sqrt(rr_new) <= tol * sqrt(bb)) { status = 0; break; }
            double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
            for (long long i = 0; i < (long long)len; i++) pv[i] = r[i] + beta * pv[i];
            rr = rr_new;
        }
        if (it > max_iter) it = max_iter;
    }
    *iters = it;
    orc_op_separable(p, kern, x, q);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)len; i++) r[i] = b[i] - q[i];
    *relres = bb > 0 ? sqrt(dot(r, r, len) / bb) : 0.0;
    free(r);
    free(pv);
    free(q);
    free(bm);
    return status;
}

/* Implicit Euler steps of u_t = Laplace(u) + g: (M + dt K) u^{k+1} = M (u^k + dt q), where q
 * holds the B-spline coefficients of the source (Eq. RitzGalerkin right-hand side with the
 * source expanded in the same basis) and M, K are the 3-D mass and stiffness operators. q may be
 * NULL (no source). Each solve starts from u^k. iters_out (length nsteps, may be NULL) receives
 * the CG iteration counts. Returns the first non-zero CG status, else 0. */
int orc_heat(const orc_problem* p, const double* kern, double* u, const double* q, int nsteps,
             double tol, int max_iter, int* iters_out, double* relres_out)
{
    if (!problem_ok(p)) return -1;
    size_t len = (size_t)p->nx * p->ny * p->nz;
    double* t = (double*)malloc(sizeof(double) * len);
    double* b = (double*)malloc(sizeof(double) * len);
    if (!t || !b) { free(t); free(b); return -3; }
    int status = 0;
    for (int s = 0; s < nsteps; s++) {
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)len; i++) t[i] = u[i] + (q ? p->dt * q[i] : 0.0);
        orc_mass(p, kern, t, b);
        int it = 0;
        double rel = 0.0;
        int st = orc_cg(p, kern, b, u, tol, max_iter, &it, &rel);
        if (iters_out) iters_out[s] = it;
        if (relres_out) relres_out[s] = rel;
        if (st != 0 && status == 0) status = st;
    }
    free(t);
    free(b);
    return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Indirect B-spline transform on tensor grids                                                 */
/* ------------------------------------------------------------------------------------------ */

/* out[kz][ky][kx] = sum_i c_i psi_i(xs[kx], ys[ky], zs[kz]) (indirect B-spline transform,
 * section 2.3), evaluated axis by axis. The mask is applied to c first. With transpose set,
 * computes instead c_i = sum_k wts_k f_k psi_i(x_k) (load vector of a function f given on the
 * grid with weights wx, wy, wz), the adjoint map used for L2 projections. */
int orc_eval_tensor(const orc_problem* p, int transpose, const double* in, int qx, const double* xs,
                    const double* wx, int qy, const double* ys, const double* wy, int qz,
                    const double* zs, const double* wz, double* out)
{
    if (!problem_ok(p)) return -1;
    int n = p->n, N[3] = {p->nx, p->ny, p->nz}, Q[3] = {qx, qy, qz};
    double h[3] = {p->hx, p->hy, p->hz};
    const double* pts[3] = {xs, ys, zs};
    const double* wts[3] = {wx, wy, wz};
    double* Bt[3];
    for (int d = 0; d < 3; d++) {
        Bt[d] = (double*)malloc(sizeof(double) * (size_t)N[d] * Q[d]);
        for (int q = 0; q < Q[d]; q++)
            for (int i = 0; i < N[d]; i++) {
                double v = psi_1d(n, N[d], h[d], i + 1, pts[d][q], 0);
                if (transpose && wts[d]) v *= wts[d][q];
                Bt[d][(size_t)q * N[d] + i] = v; /* [q][i] */
            }
    }
    /* forward: in dims N, out dims Q; transpose: in dims Q, out dims N */
    int din[3], dout[3];
    for (int d = 0; d < 3; d++) {
        din[d] = transpose ? Q[d] : N[d];
        dout[d] = transpose ? N[d] : Q[d];
    }
    size_t lin = (size_t)din[0] * din[1] * din[2];
    double* cur = (double*)malloc(sizeof(double) * lin);
    memcpy(cur, in, sizeof(double) * lin);
    if (!transpose && p->mask)
        for (size_t i = 0; i < lin; i++)
            if (!p->mask[i]) cur[i] = 0.0;
    int cd[3] = {din[0], din[1], din[2]};
    for (int axis = 0; axis < 3; axis++) {
        int nd[3] = {cd[0], cd[1], cd[2]};
        nd[axis] = dout[axis];
        double* nxt = (double*)malloc(sizeof(double) * (size_t)nd[0] * nd[1] * nd[2]);
        size_t sc = axis == 0 ? 1 : axis == 1 ? (size_t)cd[0] : (size_t)cd[0] * cd[1];
        size_t sn = axis == 0 ? 1 : axis == 1 ? (size_t)nd[0] : (size_t)nd[0] * nd[1];
#pragma omp parallel for schedule(static)
        for (int kz = 0; kz < nd[2]; kz++)
            for (int ky = 0; ky < nd[1]; ky++)
                for (int kx = 0; kx < nd[0]; kx++) {
                    int k[3] = {kx, ky, kz};
                    int o = k[axis];
                    k[axis] = 0;
                    size_t basec = ((size_t)k[2] * cd[1] + k[1]) * cd[0] + k[0];
                    double s = 0.0;
                    for (int j = 0; j < cd[axis]; j++) {
                        double bv = transpose ? Bt[axis][(size_t)j * N[axis] + o]
                                              : Bt[axis][(size_t)o * N[axis] + j];
                        s += bv * cur[basec + j * sc];
                    }
                    nxt[((size_t)kz * nd[1] + ky) * nd[0] + kx] = s;
                    (void)sn;
                }
        free(cur);
        cur = nxt;
        cd[0] = nd[0]; cd[1] = nd[1]; cd[2] = nd[2];
    }
    size_t lout = (size_t)dout[0] * dout[1] * dout[2];
    if (transpose && p->mask)
        for (size_t i = 0; i < lout; i++)
            if (!p->mask[i]) cur[i] = 0.0;
    memcpy(out, cur, sizeof(double) * lout);
    free(cur);
    for (int d = 0; d < 3; d++) free(Bt[d]);
    return 0;
}

/* 1-D quadrature rule on [0, 1] for a grid of N unknowns (the rule of the brute-force
 * assembly): returns the number of points written to xs, ws (capacity 2(N+1)(n+1)). */
int orc_axis_rule(int n, int N, double h, double* xs, double* ws)
{
    if (n < 1 || n > 7 || N < 1 || !(h > 0)) return -1;
    return axis_rule(n, N, h, xs, ws);
}

/* ------------------------------------------------------------------------------------------ */
/* Variable coefficients: Eq. RitzGalerkin / Eq. tensForm with D(x) and mu_a(x) in B-splines  */
/* ------------------------------------------------------------------------------------------ */

/* 1-D triple-product integrals on a unit grid, the per-axis factors of the tensors w^{klm} and
 * f^{klm} of Eq. tensForm. With a = k - l and b = m - l (offsets of the solution B-spline k and
 * of the coefficient B-spline m from the test B-spline l):
 *   f1[a][b] = integral beta^n(x) beta^n(x - a) beta^n(x - b) dx,
 *   w1[a][b] = integral beta^n'(x) beta^n'(x - a) beta^n(x - b) dx,
 * for a, b in [-n, n], stored at (a + n) * (2n + 1) + (b + n). Every knot of beta^n and of its
 * integer shifts is an integer or a half-integer, so between consecutive half-integers the
 * integrand is one polynomial of degree at most 3n, which (3n + 2) / 2 Gauss points integrate
 * exactly; the sum runs over the half-unit intervals of the support of beta^n(x). */
int orc_triple_kernels_1d(int n, double* f1, double* w1)
{
    if (n < 1 || n > 7) return -1;
    int L = 2 * n + 1, q = (3 * n + 2) / 2;
    double t[16], w[16];
    gauss_legendre(q, t, w);
    double half = 0.5 * (double)(n + 1);
    for (int a = -n; a <= n; a++)
        for (int b = -n; b <= n; b++) {
            double sf = 0.0, sw = 0.0;
            for (int c = 0; c < 2 * (n + 1); c++) {
                double lo = -half + 0.5 * c, hi = lo + 0.5;
                for (int g = 0; g < q; g++) {
                    double x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * t[g];
                    double wg = 0.5 * (hi - lo) * w[g];
                    double bm = orc_bspline(n, x - b);
                    sf += wg * orc_bspline(n, x) * orc_bspline(n, x - a) * bm;
                    sw += wg * orc_bspline_deriv(n, x) * orc_bspline_deriv(n, x - a) * bm;
                }
            }
            f1[(a + n) * L + (b + n)] = sf;
            w1[(a + n) * L + (b + n)] = sw;
        }
    return 0;
}

/* Coefficient fields are given at the N + 2 nodes 0..N+1 of each axis (the box faces included;
 * unknown i of the solution sits at node i + 1) and are extended evenly across the faces:
 * node -e takes the value of node e and node N+1+e that of node N+1-e, so that D and mu_a are
 * even about each face, the symmetry under which the integrals of odd-reflected basis
 * functions over the box equal their integrals over the whole space. Returns the source node
 * in [0, N+1]. g_plant == 3 (test hook) replaces the even extension by zero ghosts. */
static int reflect_even(int e, int N, int* zero)
{
    *zero = 0;
    if (e < 0) { e = -e; *zero = (g_plant == 3); }
    if (e > N + 1) { e = 2 * (N + 1) - e; *zero = (g_plant == 3); }
    return e;
}

/* Checks that single reflections reach every ghost: n <= N + 1 on each axis. */
static int var_ok(const orc_problem* p)
{
    return problem_ok(p) && p->n <= p->nx + 1 && p->n <= p->ny + 1 && p->n <= p->nz + 1;
}

typedef struct {
    int n, L;
    double f1[15 * 15], w1[15 * 15];
} var_tables;

static void var_tables_init(var_tables* t, int n, int absmode)
{
    t->n = n;
    t->L = 2 * n + 1;
    orc_triple_kernels_1d(n, t->f1, t->w1);
    if (absmode)
        for (int i = 0; i < t->L * t->L; i++) {
            t->f1[i] = fabs(t->f1[i]);
            t->w1[i] = fabs(t->w1[i]);
        }
}

/* y_l for one active node l = (ix, iy, iz) of the variable-coefficient operator:
 *   y_l = sum_k sum_m x~_k ( dt d~_m w^{klm} + m~_m f^{klm} ),
 *   f^{klm} = hx hy hz f1(ax,bx) f1(ay,by) f1(az,bz),
 *   w^{klm} = hx hy hz [ w1(ax,bx) f1(ay,by) f1(az,bz) / hx^2 + f1(ax,bx) w1(ay,by) f1(az,bz) / hy^2
 *                        + f1(ax,bx) f1(ay,by) w1(az,bz) / hz^2 ],
 * with a = k - l, b = m - l per axis, x~ the masked odd-reflected extension of x (as for the
 * constant-coefficient operator) and d~, m~ the even extensions of the coefficient fields. The
 * sum is the plain double sum over the (k, m) pairs of the support (Eq. tensForm, the
 * on-the-fly strategy of section 2.4). x is read as float (x_is_f32) or double; with absmode
 * every factor is replaced by its absolute value. */
static double var_point(const orc_problem* p, const var_tables* t, const double* d, const double* m,
                        const void* x, int x_is_f32, int ix, int iy, int iz, int absmode)
{
    int n = p->n, L = t->L;
    int N[3] = {p->nx, p->ny, p->nz}, I[3] = {ix, iy, iz};
    int cpx = p->nx + 2, cpy = p->ny + 2;   /* coefficient field pitches */
    /* per axis and offset o in [-n, n]: source of the solution (odd) and coefficient (even) */
    int xs[3][15], xsg[3][15], cs[3][15], cz[3][15];
    for (int ax = 0; ax < 3; ax++)
        for (int o = -n; o <= n; o++) {
            int src = 0;
            xsg[ax][o + n] = reflect(I[ax] + o, N[ax], &src);
            xs[ax][o + n] = src;
            cs[ax][o + n] = reflect_even(I[ax] + o + 1, N[ax], &cz[ax][o + n]);
        }
    const float* xf = (const float*)x;
    const double* xd = (const double*)x;
    double vol = p->hx * p->hy * p->hz, dt = absmode ? fabs(p->dt) : p->dt;
    double ihx2 = 1.0 / (p->hx * p->hx), ihy2 = 1.0 / (p->hy * p->hy), ihz2 = 1.0 / (p->hz * p->hz);
    double s = 0.0;
    for (int az = -n; az <= n; az++) {
        int sgz = xsg[2][az + n];
        if (!sgz) continue;
        for (int ay = -n; ay <= n; ay++) {
            int sgy = xsg[1][ay + n];
            if (!sgy) continue;
            for (int axx = -n; axx <= n; axx++) {
                int sgx = xsg[0][axx + n];
                if (!sgx) continue;
                size_t src = ((size_t)xs[2][az + n] * p->ny + xs[1][ay + n]) * p->nx + xs[0][axx + n];
                if (p->mask && !p->mask[src]) continue;
                double xv = (x_is_f32 ? (double)xf[src] : xd[src]) * (sgz * sgy * sgx);
                if (absmode) xv = fabs(xv);
                if (xv == 0.0) continue;
                for (int bz = -n; bz <= n; bz++) {
                    double fz = t->f1[(az + n) * L + (bz + n)], wz = t->w1[(az + n) * L + (bz + n)];
                    if (fz == 0.0 && wz == 0.0) continue;
                    for (int by = -n; by <= n; by++) {
                        double fy = t->f1[(ay + n) * L + (by + n)], wy = t->w1[(ay + n) * L + (by + n)];
                        if (fy == 0.0 && wy == 0.0) continue;
                        for (int bx = -n; bx <= n; bx++) {
                            double fxx = t->f1[(axx + n) * L + (bx + n)];
                            double wx = t->w1[(axx + n) * L + (bx + n)];
                            if (fxx == 0.0 && wx == 0.0) continue;
                            size_t cm = ((size_t)cs[2][bz + n] * cpy + cs[1][by + n]) * cpx + cs[0][bx + n];
                            int zero = cz[2][bz + n] || cz[1][by + n] || cz[0][bx + n];
                            double dv = zero ? 0.0 : d[cm], mv = zero ? 0.0 : m[cm];
                            if (absmode) { dv = fabs(dv); mv = fabs(mv); }
                            double wf = vol * fxx * fy * fz;
                            double ww = vol * (wx * fy * fz * ihx2 + fxx * wy * fz * ihy2 + fxx * fy * wz * ihz2);
                            s += xv * (dt * dv * ww + mv * wf);
                        }
                    }
                }
            }
        }
    }
    return s;
}

static int op_var(const orc_problem* p, const double* d, const double* m, const double* x,
                  double* y, int absmode)
{
    if (!var_ok(p)) return -1;
    var_tables t;
    var_tables_init(&t, p->n, absmode);
    size_t ntot = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long I = 0; I < (long long)ntot; I++) {
        int ix = (int)(I % p->nx), iy = (int)((I / p->nx) % p->ny);
        int iz = (int)(I / ((long long)p->nx * p->ny));
        y[I] = (p->mask && !p->mask[I]) ? 0.0 : var_point(p, &t, d, m, x, 0, ix, iy, iz, absmode);
    }
    return 0;
}

/* y = mask o A(d, m) (mask o x); d and m are (nz+2)(ny+2)(nx+2) nodal fields, x fastest. */
int orc_op_var(const orc_problem* p, const double* d, const double* m, const double* x, double* y)
{
    return op_var(p, d, m, x, y, 0);
}

/* (|A(d, m)| |x|): every triple product, coefficient and ghost-extended value replaced by its
 * absolute value; the scale of the terms summed into each output (error measure). */
int orc_abs_op_var(const orc_problem* p, const double* d, const double* m, const double* x, double* y)
{
    return op_var(p, d, m, x, y, 1);
}

/* The same definition at selected flat indices only; x read as float or double; with absmode
 * the |A(d, m)| |x| scale at those points. */
int orc_op_var_points(const orc_problem* p, const double* d, const double* m, const void* x,
                      int x_is_f32, int absmode, long long npts, const long long* pts, double* out)
{
    if (!var_ok(p)) return -1;
    var_tables t;
    var_tables_init(&t, p->n, absmode);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long k = 0; k < npts; k++) {
        long long I = pts[k];
        int ix = (int)(I % p->nx), iy = (int)((I / p->nx) % p->ny);
        int iz = (int)(I / ((long long)p->nx * p->ny));
        out[k] = (p->mask && !p->mask[I]) ? 0.0 : var_point(p, &t, d, m, x, x_is_f32, ix, iy, iz, absmode);
    }
    return 0;
}

/* 1-D coefficient basis: the B-spline centred at node e (position e h) plus its distinct mirror
 * images in both faces (even, 2(N+1)h-periodic extension), e = 0..N+1. */
static double phi_1d(int n, int N, double h, int e, double x)
{
    double u = x / h, s = 0.0;
    for (int k = -1; k <= 1; k++) {
        double shift = 2.0 * k * (N + 1);
        s += orc_bspline(n, u - e - shift);
        if (e != 0 && e != N + 1) s += orc_bspline(n, u + e - shift);
    }
    return s;
}

/* Brute-force reference for the variable-coefficient operator on tiny grids:
 *   y_i = integral over [0,1]^3 of dt D grad psi_i . grad u_h + mu_a psi_i u_h  (active i),
 *   u_h = sum_j x_j psi_j over active j,  D = sum_e d_e phi_e,  mu_a = sum_e m_e phi_e,
 * (Eq. RitzGalerkin without the boundary term) by Gauss quadrature on the tensor grid of
 * half-cells with (3n + 2) / 2 points each, every function evaluated pointwise from its
 * definition (psi_1d, phi_1d): no kernels, no ghost arrays. */
int orc_bruteforce_apply_var(const orc_problem* p, const double* d, const double* m,
                             const double* x, double* y)
{
    if (!var_ok(p)) return -1;
    int n = p->n, N[3] = {p->nx, p->ny, p->nz}, q = (3 * n + 2) / 2;
    double h[3] = {p->hx, p->hy, p->hz};
    double t[16], w[16];
    gauss_legendre(q, t, w);
    double *X[3], *W[3], *PS[3], *DP[3], *PH[3];
    int nq[3];
    for (int a = 0; a < 3; a++) {
        nq[a] = 2 * (N[a] + 1) * q;
        X[a] = (double*)malloc(sizeof(double) * nq[a]);
        W[a] = (double*)malloc(sizeof(double) * nq[a]);
        PS[a] = (double*)malloc(sizeof(double) * (size_t)nq[a] * N[a]);
        DP[a] = (double*)malloc(sizeof(double) * (size_t)nq[a] * N[a]);
        PH[a] = (double*)malloc(sizeof(double) * (size_t)nq[a] * (N[a] + 2));
        for (int c = 0; c < 2 * (N[a] + 1); c++) {
            double lo = 0.5 * h[a] * c, hi = lo + 0.5 * h[a];
            for (int g = 0; g < q; g++) {
                X[a][c * q + g] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * t[g];
                W[a][c * q + g] = 0.5 * (hi - lo) * w[g];
            }
        }
        for (int k = 0; k < nq[a]; k++) {
            for (int i = 0; i < N[a]; i++) {
                PS[a][(size_t)k * N[a] + i] = psi_1d(n, N[a], h[a], i + 1, X[a][k], 0);
                DP[a][(size_t)k * N[a] + i] = psi_1d(n, N[a], h[a], i + 1, X[a][k], 1);
            }
            for (int e = 0; e <= N[a] + 1; e++)
                PH[a][(size_t)k * (N[a] + 2) + e] = phi_1d(n, N[a], h[a], e, X[a][k]);
        }
    }
    size_t ntot = (size_t)N[0] * N[1] * N[2];
    size_t npt = (size_t)nq[0] * nq[1] * nq[2];
    /* point values: fluxes dt D grad u (3) and mu u, times the quadrature weight */
    double* F = (double*)malloc(sizeof(double) * npt * 4);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long P = 0; P < (long long)npt; P++) {
        int kx = (int)(P % nq[0]), ky = (int)((P / nq[0]) % nq[1]), kz = (int)(P / ((size_t)nq[0] * nq[1]));
        double u = 0, ux = 0, uy = 0, uz = 0, Dv = 0, Mv = 0;
        for (size_t J = 0; J < ntot; J++) {
            if (p->mask && !p->mask[J]) continue;
            int jx = (int)(J % N[0]), jy = (int)((J / N[0]) % N[1]), jz = (int)(J / ((size_t)N[0] * N[1]));
            double bx = PS[0][(size_t)kx * N[0] + jx], by = PS[1][(size_t)ky * N[1] + jy];
            double bz = PS[2][(size_t)kz * N[2] + jz];
            double gx = DP[0][(size_t)kx * N[0] + jx], gy = DP[1][(size_t)ky * N[1] + jy];
            double gz = DP[2][(size_t)kz * N[2] + jz];
            u += x[J] * bx * by * bz;
            ux += x[J] * gx * by * bz;
            uy += x[J] * bx * gy * bz;
            uz += x[J] * bx * by * gz;
        }
        for (int ez = 0; ez < N[2] + 2; ez++)
            for (int ey = 0; ey < N[1] + 2; ey++)
                for (int ex = 0; ex < N[0] + 2; ex++) {
                    size_t e = ((size_t)ez * (N[1] + 2) + ey) * (N[0] + 2) + ex;
                    double ph = PH[0][(size_t)kx * (N[0] + 2) + ex] * PH[1][(size_t)ky * (N[1] + 2) + ey] *
                                PH[2][(size_t)kz * (N[2] + 2) + ez];
                    Dv += d[e] * ph;
                    Mv += m[e] * ph;
                }
        double wq = W[0][kx] * W[1][ky] * W[2][kz];
        F[P * 4 + 0] = wq * p->dt * Dv * ux;
        F[P * 4 + 1] = wq * p->dt * Dv * uy;
        F[P * 4 + 2] = wq * p->dt * Dv * uz;
        F[P * 4 + 3] = wq * Mv * u;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (long long I = 0; I < (long long)ntot; I++) {
        if (p->mask && !p->mask[I]) { y[I] = 0.0; continue; }
        int ix = (int)(I % N[0]), iy = (int)((I / N[0]) % N[1]), iz = (int)(I / ((size_t)N[0] * N[1]));
        double s = 0.0;
        for (size_t P = 0; P < npt; P++) {
            int kx = (int)(P % nq[0]), ky = (int)((P / nq[0]) % nq[1]), kz = (int)(P / ((size_t)nq[0] * nq[1]));
            double bx = PS[0][(size_t)kx * N[0] + ix], by = PS[1][(size_t)ky * N[1] + iy];
            double bz = PS[2][(size_t)kz * N[2] + iz];
            if (bx == 0.0 || by == 0.0 || bz == 0.0) {
                double gx = DP[0][(size_t)kx * N[0] + ix], gy = DP[1][(size_t)ky * N[1] + iy];
                double gz = DP[2][(size_t)kz * N[2] + iz];
                if ((bx == 0.0 && gx == 0.0) || (by == 0.0 && gy == 0.0) || (bz == 0.0 && gz == 0.0))
                    continue;
            }
            double gx = DP[0][(size_t)kx * N[0] + ix], gy = DP[1][(size_t)ky * N[1] + iy];
            double gz = DP[2][(size_t)kz * N[2] + iz];
            s += F[P * 4 + 0] * gx * by * bz + F[P * 4 + 1] * bx * gy * bz +
                 F[P * 4 + 2] * bx * by * gz + F[P * 4 + 3] * bx * by * bz;
        }
        y[I] = s;
    }
    free(F);
    for (int a = 0; a < 3; a++) { free(X[a]); free(W[a]); free(PS[a]); free(DP[a]); free(PH[a]); }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Robin (boundary penalty) problems on the box: the untruncated B-spline basis                */
/* ------------------------------------------------------------------------------------------ */

/* With the boundary penalty method (section 3, Dirichlet data approximated by a Robin condition
 * weighted by a penalty; the boundary integral of Eq. RitzGalerkin) the basis does not vanish on
 * the faces: every B-spline beta(x/h - i) whose support meets the box (0, (N+1)h) is an unknown,
 * i = i0 .. N+1-i0 with i0 = -floor(n/2), i.e. Nt = N + 2 + 2 floor(n/2) per axis, array
 * position a = i - i0. */
int orc_robin_size(int n, int N) { return N + 2 + 2 * (n / 2); }

/* Dense Nt x Nt factors of one axis, integrals truncated to the box [0, (N+1)h]:
 *   M_ab = int beta_a beta_b dx,  K_ab = int beta_a' beta_b' dx,
 *   E_ab = beta_a(0) beta_b(0) + beta_a((N+1)h) beta_b((N+1)h)   (the two faces of the axis).
 * Quadrature: n + 1 Gauss points per half-cell of the box (the rule of the brute-force matrix),
 * exact for the degree-2n products. */
int orc_robin_1d(int n, int N, double h, double* M, double* K, double* E)
{
    if (n < 1 || n > 7 || N < 1 || !(h > 0)) return -1;
    int Nt = orc_robin_size(n, N), i0 = -(n / 2);
    int cap = 2 * (N + 1) * (n + 1);
    double* xs = (double*)malloc(sizeof(double) * cap);
    double* ws = (double*)malloc(sizeof(double) * cap);
    int nq = axis_rule(n, N, h, xs, ws);
    for (int a = 0; a < Nt; a++)
        for (int b = 0; b < Nt; b++) {
            double sm = 0.0, sk = 0.0;
            for (int q = 0; q < nq; q++) {
                double u = xs[q] / h;
                sm += ws[q] * orc_bspline(n, u - (a + i0)) * orc_bspline(n, u - (b + i0));
                sk += ws[q] * orc_bspline_deriv(n, u - (a + i0)) * orc_bspline_deriv(n, u - (b + i0)) / (h * h);
            }
            M[a * Nt + b] = sm;
            K[a * Nt + b] = sk;
            E[a * Nt + b] = orc_bspline(n, 0.0 - (a + i0)) * orc_bspline(n, 0.0 - (b + i0)) +
                            (g_plant == 4 ? 0.0 :   /* test hook: the far face left out */
                             orc_bspline(n, (double)(N + 1) - (a + i0)) * orc_bspline(n, (double)(N + 1) - (b + i0)));
        }
    free(xs);
    free(ws);
    return 0;
}

typedef struct {
    int Nt[3];
    double *M[3], *K[3], *E[3];
} robin_tabs;

static void robin_free(robin_tabs* t)
{
    for (int d = 0; d < 3; d++) { free(t->M[d]); free(t->K[d]); free(t->E[d]); }
}

static int robin_init(const orc_problem* p, robin_tabs* t, int absmode)
{
    int N[3] = {p->nx, p->ny, p->nz};
    double h[3] = {p->hx, p->hy, p->hz};
    for (int d = 0; d < 3; d++) {
        int Nt = orc_robin_size(p->n, N[d]);
        t->Nt[d] = Nt;
        t->M[d] = (double*)malloc(sizeof(double) * Nt * Nt);
        t->K[d] = (double*)malloc(sizeof(double) * Nt * Nt);
        t->E[d] = (double*)malloc(sizeof(double) * Nt * Nt);
        if (orc_robin_1d(p->n, N[d], h[d], t->M[d], t->K[d], t->E[d])) return -1;
        if (absmode)
            for (int i = 0; i < Nt * Nt; i++) {
                t->M[d][i] = fabs(t->M[d][i]);
                t->K[d][i] = fabs(t->K[d][i]);
                t->E[d][i] = fabs(t->E[d][i]);
            }
    }
    return 0;
}

/* Weight of unknown k in output l of the Robin operator from the 1-D factors. */
static double robin_weight(const robin_tabs* t, double dt, double pen, const int* l, const int* k)
{
    double m[3], s[3], e[3];
    for (int d = 0; d < 3; d++) {
        size_t o = (size_t)l[d] * t->Nt[d] + k[d];
        m[d] = t->M[d][o];
        s[d] = t->K[d][o];
        e[d] = t->E[d][o];
    }
    return m[2] * m[1] * m[0] + dt * (s[2] * m[1] * m[0] + m[2] * s[1] * m[0] + m[2] * m[1] * s[0]) +
           pen * (e[2] * m[1] * m[0] + m[2] * e[1] * m[0] + m[2] * m[1] * e[0]);
}

/* y = A_R x on the Nt^3 unknowns of the Robin basis (problem nx, ny, nz = interior nodes N of
 * the box):
 *   A_R = Mz My Mx + dt (Kz My Mx + Mz Ky Mx + Mz My Kx) + pen (Ez My Mx + Mz Ey Mx + Mz My Ex),
 * Eq. RitzGalerkin with D = dt, mu_a = 1 and the boundary term weighted by pen (1/(2 gamma) in
 * the paper's notation), summed directly over the (2n+1)^3 band of each output. No mask. */
static int op_robin(const orc_problem* p, double pen, const double* x, double* y, int absmode)
{
    if (!problem_ok(p) || p->mask) return -1;
    robin_tabs t;
    memset(&t, 0, sizeof t);
    if (robin_init(p, &t, absmode)) { robin_free(&t); return -1; }
    int n = p->n, *Nt = t.Nt;
    double dt = absmode ? fabs(p->dt) : p->dt, pw = absmode ? fabs(pen) : pen;
    size_t len = (size_t)Nt[0] * Nt[1] * Nt[2];
#pragma omp parallel for schedule(dynamic, 64)
    for (long long I = 0; I < (long long)len; I++) {
        int l[3] = {(int)(I % Nt[0]), (int)((I / Nt[0]) % Nt[1]), (int)(I / ((long long)Nt[0] * Nt[1]))};
        double s = 0.0;
        for (int kz = l[2] - n; kz <= l[2] + n; kz++) {
            if (kz < 0 || kz >= Nt[2]) continue;
            for (int ky = l[1] - n; ky <= l[1] + n; ky++) {
                if (ky < 0 || ky >= Nt[1]) continue;
                for (int kx = l[0] - n; kx <= l[0] + n; kx++) {
                    if (kx < 0 || kx >= Nt[0]) continue;
                    int k[3] = {kx, ky, kz};
                    double xv = x[((size_t)kz * Nt[1] + ky) * Nt[0] + kx];
                    s += robin_weight(&t, dt, pw, l, k) * (absmode ? fabs(xv) : xv);
                }
            }
        }
        y[I] = s;
    }
    robin_free(&t);
    return 0;
}

int orc_op_robin(const orc_problem* p, double pen, const double* x, double* y)
{
    return op_robin(p, pen, x, y, 0);
}

int orc_abs_op_robin(const orc_problem* p, double pen, const double* x, double* y)
{
    return op_robin(p, pen, x, y, 1);
}

/* Brute-force reference for A_R on tiny grids: the volume integral of u psi_i + dt grad u . grad
 * psi_i over the box on the tensor half-cell Gauss grid, plus pen times the surface integral of
 * u psi_i over the six faces on the 2-D half-cell Gauss grid of each face, with u and every
 * B-spline evaluated pointwise (no 1-D factors, no bands). */
int orc_bruteforce_apply_robin(const orc_problem* p, double pen, const double* x, double* y)
{
    if (!problem_ok(p) || p->mask) return -1;
    int n = p->n, N[3] = {p->nx, p->ny, p->nz}, Nt[3], i0 = -(n / 2);
    double h[3] = {p->hx, p->hy, p->hz}, L[3];
    double *X[3], *W[3], *B[3], *G[3], *F0[3], *F1[3];
    int nq[3];
    for (int a = 0; a < 3; a++) {
        Nt[a] = orc_robin_size(n, N[a]);
        L[a] = (N[a] + 1) * h[a];
        int cap = 2 * (N[a] + 1) * (n + 1);
        X[a] = (double*)malloc(sizeof(double) * cap);
        W[a] = (double*)malloc(sizeof(double) * cap);
        nq[a] = axis_rule(n, N[a], h[a], X[a], W[a]);
        B[a] = (double*)malloc(sizeof(double) * (size_t)nq[a] * Nt[a]);
        G[a] = (double*)malloc(sizeof(double) * (size_t)nq[a] * Nt[a]);
        F0[a] = (double*)malloc(sizeof(double) * Nt[a]);
        F1[a] = (double*)malloc(sizeof(double) * Nt[a]);
        for (int i = 0; i < Nt[a]; i++) {
            for (int q = 0; q < nq[a]; q++) {
                double u = X[a][q] / h[a] - (i + i0);
                B[a][(size_t)q * Nt[a] + i] = orc_bspline(n, u);
                G[a][(size_t)q * Nt[a] + i] = orc_bspline_deriv(n, u) / h[a];
            }
            F0[a][i] = orc_bspline(n, 0.0 / h[a] - (i + i0));
            F1[a][i] = orc_bspline(n, L[a] / h[a] - (i + i0));
        }
    }
    size_t len = (size_t)Nt[0] * Nt[1] * Nt[2];
    memset(y, 0, sizeof(double) * len);
    /* volume: point values of u and grad u, then the projection onto every basis function */
    size_t npt = (size_t)nq[0] * nq[1] * nq[2];
    double* U = (double*)malloc(sizeof(double) * npt * 4);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long P = 0; P < (long long)npt; P++) {
        int q[3] = {(int)(P % nq[0]), (int)((P / nq[0]) % nq[1]), (int)(P / ((size_t)nq[0] * nq[1]))};
        double u = 0, gx = 0, gy = 0, gz = 0;
        for (size_t J = 0; J < len; J++) {
            int j[3] = {(int)(J % Nt[0]), (int)((J / Nt[0]) % Nt[1]), (int)(J / ((size_t)Nt[0] * Nt[1]))};
            double b0 = B[0][(size_t)q[0] * Nt[0] + j[0]], b1 = B[1][(size_t)q[1] * Nt[1] + j[1]];
            double b2 = B[2][(size_t)q[2] * Nt[2] + j[2]];
            if (b0 == 0.0 && G[0][(size_t)q[0] * Nt[0] + j[0]] == 0.0) continue;
            double g0 = G[0][(size_t)q[0] * Nt[0] + j[0]], g1 = G[1][(size_t)q[1] * Nt[1] + j[1]];
            double g2 = G[2][(size_t)q[2] * Nt[2] + j[2]];
            u += x[J] * b0 * b1 * b2;
            gx += x[J] * g0 * b1 * b2;
            gy += x[J] * b0 * g1 * b2;
            gz += x[J] * b0 * b1 * g2;
        }
        double w = W[0][q[0]] * W[1][q[1]] * W[2][q[2]];
        U[P * 4 + 0] = w * u;
        U[P * 4 + 1] = w * p->dt * gx;
        U[P * 4 + 2] = w * p->dt * gy;
        U[P * 4 + 3] = w * p->dt * gz;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (long long I = 0; I < (long long)len; I++) {
        int i[3] = {(int)(I % Nt[0]), (int)((I / Nt[0]) % Nt[1]), (int)(I / ((size_t)Nt[0] * Nt[1]))};
        double s = 0.0;
        for (size_t P = 0; P < npt; P++) {
            int q[3] = {(int)(P % nq[0]), (int)((P / nq[0]) % nq[1]), (int)(P / ((size_t)nq[0] * nq[1]))};
            double b0 = B[0][(size_t)q[0] * Nt[0] + i[0]], b1 = B[1][(size_t)q[1] * Nt[1] + i[1]];
            double b2 = B[2][(size_t)q[2] * Nt[2] + i[2]];
            double g0 = G[0][(size_t)q[0] * Nt[0] + i[0]], g1 = G[1][(size_t)q[1] * Nt[1] + i[1]];
            double g2 = G[2][(size_t)q[2] * Nt[2] + i[2]];
            s += U[P * 4 + 0] * b0 * b1 * b2 + U[P * 4 + 1] * g0 * b1 * b2 + U[P * 4 + 2] * b0 * g1 * b2 +
                 U[P * 4 + 3] * b0 * b1 * g2;
        }
        y[I] = s;
    }
    free(U);
    /* faces: axis a fixed at 0 or L[a]; the other two axes on their Gauss grids */
    for (int a = 0; a < 3; a++) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int side = 0; side < 2; side++) {
            const double* Fa = side ? F1[a] : F0[a];
            size_t nfp = (size_t)nq[b] * nq[c];
            double* Uf = (double*)malloc(sizeof(double) * nfp);
#pragma omp parallel for schedule(dynamic, 16)
            for (long long P = 0; P < (long long)nfp; P++) {
                int qb = (int)(P % nq[b]), qc = (int)(P / nq[b]);
                double u = 0.0;
                for (size_t J = 0; J < len; J++) {
                    int j[3] = {(int)(J % Nt[0]), (int)((J / Nt[0]) % Nt[1]), (int)(J / ((size_t)Nt[0] * Nt[1]))};
                    u += x[J] * Fa[j[a]] * B[b][(size_t)qb * Nt[b] + j[b]] * B[c][(size_t)qc * Nt[c] + j[c]];
                }
                Uf[P] = W[b][qb] * W[c][qc] * u;
            }
#pragma omp parallel for schedule(dynamic, 4)
            for (long long I = 0; I < (long long)len; I++) {
                int i[3] = {(int)(I % Nt[0]), (int)((I / Nt[0]) % Nt[1]), (int)(I / ((size_t)Nt[0] * Nt[1]))};
                if (Fa[i[a]] == 0.0) continue;
                double s = 0.0;
                for (size_t P = 0; P < nfp; P++) {
                    int qb = (int)(P % nq[b]), qc = (int)(P / nq[b]);
                    s += Uf[P] * B[b][(size_t)qb * Nt[b] + i[b]] * B[c][(size_t)qc * Nt[c] + i[c]];
                }
                y[I] += pen * Fa[i[a]] * s;
            }
            free(Uf);
        }
    }
    for (int a = 0; a < 3; a++) { free(X[a]); free(W[a]); free(B[a]); free(G[a]); free(F0[a]); free(F1[a]); }
    return 0;
}

/* Diagonal of the system matrix: robin = 0, the odd-reflected (and masked) operator of
 * orc_op_stencil (A_ii is the sum of the stencil weights whose reflected source is i itself,
 * with the reflection's sign); robin = 1, A_R (products of the 1-D diagonals). The Jacobi
 * preconditioner of the paper's large run (section 3) divides by it. Inactive nodes get 1. */
int orc_diag(const orc_problem* p, double pen, int robin, double* d)
{
    if (!problem_ok(p)) return -1;
    if (robin) {
        if (p->mask) return -1;
        robin_tabs t;
        memset(&t, 0, sizeof t);
        if (robin_init(p, &t, 0)) { robin_free(&t); return -1; }
        size_t len = (size_t)t.Nt[0] * t.Nt[1] * t.Nt[2];
        for (size_t I = 0; I < len; I++) {
            int l[3] = {(int)(I % t.Nt[0]), (int)((I / t.Nt[0]) % t.Nt[1]), (int)(I / ((size_t)t.Nt[0] * t.Nt[1]))};
            d[I] = robin_weight(&t, p->dt, pen, l, l);
        }
        robin_free(&t);
        return 0;
    }
    int n = p->n, L = 2 * n + 1;
    double kern[6 * 15];
    if (orc_problem_kernels(p, kern)) return -1;
    const double *Mx = kern, *Kx = kern + L, *My = kern + 2 * L, *Ky = kern + 3 * L;
    const double *Mz = kern + 4 * L, *Kz = kern + 5 * L;
    size_t len = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long long I = 0; I < (long long)len; I++) {
        int ix = (int)(I % p->nx), iy = (int)((I / p->nx) % p->ny), iz = (int)(I / ((long long)p->nx * p->ny));
        if (p->mask && !p->mask[I]) { d[I] = 1.0; continue; }
        double s = 0.0;
        for (int c = 0; c < L; c++) {
            int sz, gz = reflect(iz + c - n, p->nz, &sz);
            if (!gz || sz != iz) continue;
            for (int b = 0; b < L; b++) {
                int sy, gy = reflect(iy + b - n, p->ny, &sy);
                if (!gy || sy != iy) continue;
                for (int a = 0; a < L; a++) {
                    int sx, gx = reflect(ix + a - n, p->nx, &sx);
                    if (!gx || sx != ix) continue;
                    double w = Mz[c] * My[b] * Mx[a] +
                               p->dt * (Kz[c] * My[b] * Mx[a] + Mz[c] * Ky[b] * Mx[a] + Mz[c] * My[b] * Kx[a]);
                    s += w * (gz * gy * gx);
                }
            }
        }
        d[I] = s;
    }
    return 0;
}

/* Jacobi-preconditioned conjugate gradient (the solver of the paper's large run, section 3):
 * textbook PCG with z = r / diag(A), for the reflected operator (robin = 0, masked) or A_R
 * (robin = 1). Stops when ||r|| <= tol ||b||; reports iterations and the true relative
 * residual. */
int orc_pcg(const orc_problem* p, double pen, int robin, const double* b, double* x, double tol,
            int max_iter, int* iters, double* relres)
{
    if (!problem_ok(p)) return -1;
    size_t len = robin ? (size_t)orc_robin_size(p->n, p->nx) * orc_robin_size(p->n, p->ny) *
                             orc_robin_size(p->n, p->nz)
                       : (size_t)p->nx * p->ny * p->nz;
    double kern[6 * 15];
    if (!robin && orc_problem_kernels(p, kern)) return -1;
    double* dg = (double*)malloc(sizeof(double) * len);
    double* r = (double*)malloc(sizeof(double) * len);
    double* z = (double*)malloc(sizeof(double) * len);
    double* pv = (double*)malloc(sizeof(double) * len);
    double* q = (double*)malloc(sizeof(double) * len);
    double* bm = (double*)malloc(sizeof(double) * len);
    if (!dg || !r || !z || !pv || !q || !bm || orc_diag(p, pen, robin, dg)) {
        free(dg); free(r); free(z); free(pv); free(q); free(bm);
        return -1;
    }
    for (size_t i = 0; i < len; i++) {
        int act = robin || !p->mask || p->mask[i];
        bm[i] = act ? b[i] : 0.0;
        if (!act) x[i] = 0.0;
    }
#define APPLY(in, out) (robin ? orc_op_robin(p, pen, in, out) : orc_op_separable(p, kern, in, out))
    double bb = dot(bm, bm, len);
    APPLY(x, q);
    for (size_t i = 0; i < len; i++) { r[i] = bm[i] - q[i]; z[i] = r[i] / dg[i]; pv[i] = z[i]; }
    double rz = dot(r, z, len), rr = dot(r, r, len);
    int status = 1, it = 0;
    if (bb == 0.0) {
        memset(x, 0, sizeof(double) * len);
        status = 0;
    } else if (sqrt(rr) <= tol * sqrt(bb)) {
        status = 0;
    } else {
        for (it = 1; it <= max_iter; it++) {
            APPLY(pv, q);
            double pq = dot(pv, q, len);
            if (!(pq > 0.0)) { status = -5; break; }
            double alpha = rz / pq;
            for (size_t i = 0; i < len; i++) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }
            rr = dot(r, r, len);
            if (sqrt(rr) <= tol * sqrt(bb)) { status = 0; break; }
            for (size_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
            double rz_new = dot(r, z, len);
            double beta = rz_new / rz;
            for (size_t i = 0; i < len; i++) pv[i] = z[i] + beta * pv[i];
            rz = rz_new;
        }
        if (it > max_iter) it = max_iter;
    }
    *iters = it;
    APPLY(x, q);
    for (size_t i = 0; i < len; i++) r[i] = bm[i] - q[i];
    *relres = bb > 0 ? sqrt(dot(r, r, len) / bb) : 0.0;
#undef APPLY
    free(dg); free(r); free(z); free(pv); free(q); free(bm);
    return status;
}

/* 1-D transfer between the Robin bases of two grids on the same interval [0, L],
 * L = (Nf+1) hf = (Nc+1) hc:  T_fc = int_0^L beta(x/hf - f) beta(x/hc - c) dx (dense Ntf x Ntc).
 * The integrand is a polynomial of degree 2n between consecutive breakpoints of either grid (the
 * half-multiples of hf and of hc), so n + 1 Gauss points per piece integrate it exactly. */
int orc_transfer_1d(int n, int Nf, double hf, int Nc, double hc, double* T)
{
    if (n < 1 || n > 7 || Nf < 1 || Nc < 1 || !(hf > 0) || !(hc > 0)) return -1;
    double L = (Nf + 1) * hf;
    if (fabs((Nc + 1) * hc - L) > 1e-12 * L) return -1;
    int Ntf = orc_robin_size(n, Nf), Ntc = orc_robin_size(n, Nc), i0 = -(n / 2);
    int nbf = 2 * (Nf + 1), nbc = 2 * (Nc + 1), nb = 0;
    double* br = (double*)malloc(sizeof(double) * (nbf + nbc + 2));
    for (int k = 0; k <= nbf; k++) br[nb++] = 0.5 * hf * k;
    for (int k = 0; k <= nbc; k++) br[nb++] = 0.5 * hc * k;
    for (int i = 1; i < nb; i++)   /* insertion sort */
        for (int j = i; j > 0 && br[j - 1] > br[j]; j--) { double t = br[j]; br[j] = br[j - 1]; br[j - 1] = t; }
    double t[16], w[16];
    gauss_legendre(n + 1, t, w);
    memset(T, 0, sizeof(double) * (size_t)Ntf * Ntc);
    for (int s = 0; s + 1 < nb; s++) {
        double a = br[s], b = br[s + 1];
        if (!(b - a > 1e-14 * L)) continue;
        for (int g = 0; g <= n; g++) {
            double x = 0.5 * (a + b) + 0.5 * (b - a) * t[g], wg = 0.5 * (b - a) * w[g];
            for (int f = 0; f < Ntf; f++) {
                double vf = orc_bspline(n, x / hf - (f + i0));
                if (vf == 0.0) continue;
                for (int c = 0; c < Ntc; c++)
                    T[(size_t)f * Ntc + c] += wg * vf * orc_bspline(n, x / hc - (c + i0));
            }
        }
    }
    free(br);
    return 0;
}

/* Solves the dense system A X = B (A n x n, B n x m, both row-major, overwritten) by Gaussian
 * elimination with partial pivoting; X is left in B. */
static int dense_solve(int n, int m, double* A, double* B)
{
    for (int k = 0; k < n; k++) {
        int piv = k;
        for (int i = k + 1; i < n; i++) if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (A[piv * n + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; j++) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            for (int j = 0; j < m; j++) { double t = B[k * m + j]; B[k * m + j] = B[piv * m + j]; B[piv * m + j] = t; }
        }
        for (int i = k + 1; i < n; i++) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
            for (int j = 0; j < m; j++) B[i * m + j] -= f * B[k * m + j];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        for (int j = 0; j < m; j++) {
            double s = B[k * m + j];
            for (int i = k + 1; i < n; i++) s -= A[k * n + i] * B[i * m + j];
            B[k * m + j] = s / A[k * n + k];
        }
    }
    return 0;
}

/* L2 projection of a coarse Robin expansion onto the fine Robin basis of the same box (the
 * coarse-grid initialisation of the paper's large run, section 3): xf = M_f^{-1} T xc, with the
 * fine Gram matrix and the transfer factorising per axis, so xf = (Pz Py Px) xc with
 * P_d = M_d^{-1} T_d (dense 1-D solves). fine / coarse: problems with nx, ny, nz = interior nodes. */
int orc_prolong_robin(const orc_problem* fine, const orc_problem* coarse, const double* xc, double* xf)
{
    if (!problem_ok(fine) || !problem_ok(coarse) || fine->n != coarse->n) return -1;
    int n = fine->n;
    int Nf[3] = {fine->nx, fine->ny, fine->nz}, Nc[3] = {coarse->nx, coarse->ny, coarse->nz};
    double hf[3] = {fine->hx, fine->hy, fine->hz}, hc[3] = {coarse->hx, coarse->hy, coarse->hz};
    int tf[3], tc[3];
    double* P[3];
    for (int d = 0; d < 3; d++) {
        tf[d] = orc_robin_size(n, Nf[d]);
        tc[d] = orc_robin_size(n, Nc[d]);
        double* M = (double*)malloc(sizeof(double) * tf[d] * tf[d]);
        double* K = (double*)malloc(sizeof(double) * tf[d] * tf[d]);
        double* E = (double*)malloc(sizeof(double) * tf[d] * tf[d]);
        P[d] = (double*)malloc(sizeof(double) * (size_t)tf[d] * tc[d]);
        int rc = orc_robin_1d(n, Nf[d], hf[d], M, K, E);
        if (!rc) rc = orc_transfer_1d(n, Nf[d], hf[d], Nc[d], hc[d], P[d]);
        if (!rc) rc = dense_solve(tf[d], tc[d], M, P[d]);
        free(M); free(K); free(E);
        if (rc) { for (int e = 0; e <= d; e++) free(P[e]); return -1; }
    }
    /* apply P along x, then y, then z */
    size_t s1 = (size_t)tf[0] * tc[1] * tc[2], s2 = (size_t)tf[0] * tf[1] * tc[2];
    double* t1 = (double*)calloc(s1, sizeof(double));
    double* t2 = (double*)calloc(s2, sizeof(double));
    for (int z = 0; z < tc[2]; z++)
        for (int y = 0; y < tc[1]; y++)
            for (int f = 0; f < tf[0]; f++) {
                double s = 0.0;
                for (int c = 0; c < tc[0]; c++) s += P[0][(size_t)f * tc[0] + c] * xc[((size_t)z * tc[1] + y) * tc[0] + c];
                t1[((size_t)z * tc[1] + y) * tf[0] + f] = s;
            }
    for (int z = 0; z < tc[2]; z++)
        for (int f = 0; f < tf[1]; f++)
            for (int x = 0; x < tf[0]; x++) {
                double s = 0.0;
                for (int c = 0; c < tc[1]; c++) s += P[1][(size_t)f * tc[1] + c] * t1[((size_t)z * tc[1] + c) * tf[0] + x];
                t2[((size_t)z * tf[1] + f) * tf[0] + x] = s;
            }
    for (int f = 0; f < tf[2]; f++)
        for (int y = 0; y < tf[1]; y++)
            for (int x = 0; x < tf[0]; x++) {
                double s = 0.0;
                for (int c = 0; c < tc[2]; c++) s += P[2][(size_t)f * tc[2] + c] * t2[((size_t)c * tf[1] + y) * tf[0] + x];
                xf[((size_t)f * tf[1] + y) * tf[0] + x] = s;
            }
    free(t1); free(t2);
    for (int d = 0; d < 3; d++) free(P[d]);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Jacobi preconditioning of the variable-coefficient operator                                 */
/* ------------------------------------------------------------------------------------------ */

/* Diagonal of A(d, m): A_ll = (A(d, m) e_l)_l, each entry evaluated from the triple-sum definition
 * of var_point with x = e_l (whose odd-reflected extension carries the row's own mirror images).
 * Inactive nodes get 1. */
int orc_diag_var(const orc_problem* p, const double* d, const double* m, double* dg)
{
    if (!var_ok(p)) return -1;
    var_tables t;
    var_tables_init(&t, p->n, 0);
    size_t len = (size_t)p->nx * p->ny * p->nz;
    int failed = 0;
#pragma omp parallel
    {
        double* e = (double*)calloc(len, sizeof(double));
        if (!e) failed = 1;
#pragma omp for schedule(dynamic, 16)
        for (long long I = 0; I < (long long)len; I++) {
            if (!e) continue;
            if (p->mask && !p->mask[I]) { dg[I] = 1.0; continue; }
            int ix = (int)(I % p->nx), iy = (int)((I / p->nx) % p->ny);
            int iz = (int)(I / ((long long)p->nx * p->ny));
            e[I] = 1.0;
            dg[I] = var_point(p, &t, d, m, e, 0, ix, iy, iz, 0);
            e[I] = 0.0;
        }
        free(e);
    }
    return failed ? -3 : 0;
}

/* Jacobi-preconditioned CG on A(d, m) x = b (textbook PCG, z = r / diag), masked. */
int orc_pcg_var(const orc_problem* p, const double* d, const double* m, const double* b, double* x,
                double tol, int max_iter, int* iters, double* relres)
{
    if (!var_ok(p)) return -1;
    size_t len = (size_t)p->nx * p->ny * p->nz;
    double* dg = (double*)malloc(sizeof(double) * len);
    double* r = (double*)malloc(sizeof(double) * len);
    double* z = (double*)malloc(sizeof(double) * len);
    double* pv = (double*)malloc(sizeof(double) * len);
    double* q = (double*)malloc(sizeof(double) * len);
    double* bm = (double*)malloc(sizeof(double) * len);
    if (!dg || !r || !z || !pv || !q || !bm || orc_diag_var(p, d, m, dg)) {
        free(dg); free(r); free(z); free(pv); free(q); free(bm);
        return -1;
    }
    for (size_t i = 0; i < len; i++) {
        int act = !p->mask || p->mask[i];
        bm[i] = act ? b[i] : 0.0;
        if (!act) x[i] = 0.0;
    }
    double bb = dot(bm, bm, len);
    orc_op_var(p, d, m, x, q);
    for (size_t i = 0; i < len; i++) { r[i] = bm[i] - q[i]; z[i] = r[i] / dg[i]; pv[i] = z[i]; }
    double rz = dot(r, z, len), rr = dot(r, r, len);
    int status = 1, it = 0;
    if (bb == 0.0) {
        memset(x, 0, sizeof(double) * len);
        status = 0;
    } else if (sqrt(rr) <= tol * sqrt(bb)) {
        status = 0;
    } else {
        for (it = 1; it <= max_iter; it++) {
            orc_op_var(p, d, m, pv, q);
            double pq = dot(pv, q, len);
            if (!(pq > 0.0)) { status = -5; break; }
            double alpha = rz / pq;
            for (size_t i = 0; i < len; i++) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }
            rr = dot(r, r, len);
            if (sqrt(rr) <= tol * sqrt(bb)) { status = 0; break; }
            for (size_t i = 0; i < len; i++) z[i] = r[i] / dg[i];
            double rz_new = dot(r, z, len);
            double beta = rz_new / rz;
            for (size_t i = 0; i < len; i++) pv[i] = z[i] + beta * pv[i];
            rz = rz_new;
        }
        if (it > max_iter) it = max_iter;
    }
    *iters = it;
    orc_op_var(p, d, m, x, q);
    for (size_t i = 0; i < len; i++) r[i] = bm[i] - q[i];
    *relres = bb > 0 ? sqrt(dot(r, r, len) / bb) : 0.0;
    free(dg); free(r); free(z); free(pv); free(q); free(bm);
    return status;
}

/* A_R x at selected flat indices only (the band-sum definition of orc_op_robin), x read as float
 * or double; with absmode the |A_R| |x| scale there. For parity checks at sizes where a full
 * oracle pass is too slow. */
int orc_op_robin_points(const orc_problem* p, double pen, const void* x, int x_is_f32, int absmode,
                        long long npts, const long long* pts, double* out)
{
    if (!problem_ok(p) || p->mask) return -1;
    robin_tabs t;
    memset(&t, 0, sizeof t);
    if (robin_init(p, &t, absmode)) { robin_free(&t); return -1; }
    const double dtw = absmode ? fabs(p->dt) : p->dt, penw = absmode ? fabs(pen) : pen;
    int n = p->n, *Nt = t.Nt;
    const float* xf = (const float*)x;
    const double* xd = (const double*)x;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long q = 0; q < npts; q++) {
        long long I = pts[q];
        int l[3] = {(int)(I % Nt[0]), (int)((I / Nt[0]) % Nt[1]), (int)(I / ((long long)Nt[0] * Nt[1]))};
        double s = 0.0;
        for (int kz = l[2] - n; kz <= l[2] + n; kz++) {
            if (kz < 0 || kz >= Nt[2]) continue;
            for (int ky = l[1] - n; ky <= l[1] + n; ky++) {
                if (ky < 0 || ky >= Nt[1]) continue;
                for (int kx = l[0] - n; kx <= l[0] + n; kx++) {
                    if (kx < 0 || kx >= Nt[0]) continue;
                    int k[3] = {kx, ky, kz};
                    size_t src = ((size_t)kz * Nt[1] + ky) * Nt[0] + kx;
                    double xv = x_is_f32 ? (double)xf[src] : xd[src];
                    s += robin_weight(&t, dtw, penw, l, k) * (absmode ? fabs(xv) : xv);
                }
            }
        }
        out[q] = s;
    }
    robin_free(&t);
    return 0;
}
