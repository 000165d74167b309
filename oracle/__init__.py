"""FP64 CPU oracle for the tensor B-spline heat-equation operator (arXiv:1904.03057).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA product path never
imports it, and the two share no code.

The arithmetic lives in ``bsk_oracle.c`` (plain C, double precision, OpenMP over outer loops,
``-ffp-contract=off`` so that x86 and Arm give identical results). This module compiles it with
gcc into ``oracle/_build/`` and wraps it with ctypes over numpy arrays. Each wrapper names the
passage of the paper that the C routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbsk_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("n", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("dt", ctypes.c_double), ("mask", ctypes.POINTER(ctypes.c_uint8)),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP) if missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_bspline.restype = ctypes.c_double
            L.orc_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_bspline_deriv.restype = ctypes.c_double
            L.orc_bspline_deriv.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, _D, _D]
            L.orc_kernels_1d.argtypes = [ctypes.c_int, _D, _D]
            L.orc_bspline_kernels.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
            P = ctypes.POINTER(_Problem)
            L.orc_problem_kernels.argtypes = [P, _D]
            L.orc_set_plant.argtypes = [ctypes.c_int]
            for name in ("orc_op_stencil", "orc_op_separable", "orc_mass", "orc_abs_op"):
                getattr(L, name).argtypes = [P, _D, _D, _D]
            L.orc_op_points.argtypes = [P, _D, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                        ctypes.POINTER(ctypes.c_longlong), _D]
            L.orc_bruteforce_matrix.argtypes = [P, ctypes.c_int, _D, _I]
            L.orc_dot.restype = ctypes.c_double
            L.orc_dot.argtypes = [_D, _D, ctypes.c_longlong]
            L.orc_cg.argtypes = [P, _D, _D, _D, ctypes.c_double, ctypes.c_int, _I, _D]
            L.orc_heat.argtypes = [P, _D, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   _I, _D]
            L.orc_eval_tensor.argtypes = [P, ctypes.c_int, _D, ctypes.c_int, _D, _D,
                                          ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D]
            L.orc_axis_rule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
            L.orc_triple_kernels_1d.argtypes = [ctypes.c_int, _D, _D]
            L.orc_robin_size.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_robin_1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D]
            for name in ("orc_op_robin", "orc_abs_op_robin", "orc_bruteforce_apply_robin"):
                getattr(L, name).argtypes = [P, ctypes.c_double, _D, _D]
            L.orc_diag.argtypes = [P, ctypes.c_double, ctypes.c_int, _D]
            L.orc_pcg.argtypes = [P, ctypes.c_double, ctypes.c_int, _D, _D, ctypes.c_double,
                                  ctypes.c_int, _I, _D]
            L.orc_transfer_1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_double, _D]
            L.orc_prolong_robin.argtypes = [P, P, _D, _D]
            L.orc_diag_var.argtypes = [P, _D, _D, _D]
            L.orc_op_robin_points.argtypes = [P, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_longlong,
                                              ctypes.POINTER(ctypes.c_longlong), _D]
            L.orc_pcg_var.argtypes = [P, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _I, _D]
            for name in ("orc_op_var", "orc_abs_op_var", "orc_bruteforce_apply_var"):
                getattr(L, name).argtypes = [P, _D, _D, _D, _D]
            L.orc_op_var_points.argtypes = [P, _D, _D, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong), _D]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Grid of nx*ny*nz unknowns (array layout [nz][ny][nx]), degree n, steps h, weight dt of
    the stiffness term, optional uint8 node mask. Faces carry zero Dirichlet data by odd
    reflection; masked-out nodes are removed from the system (principal submatrix)."""

    def __init__(self, nx, ny, nz, n, hx, hy=None, hz=None, dt=0.0, mask=None):
        self.nx, self.ny, self.nz, self.n = int(nx), int(ny), int(nz), int(n)
        self.hx = float(hx)
        self.hy = float(hx if hy is None else hy)
        self.hz = float(hx if hz is None else hz)
        self.dt = float(dt)
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        if self.mask is not None:
            assert self.mask.shape == (self.nz, self.ny, self.nx)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def _c(self):
        s = _Problem(self.nx, self.ny, self.nz, self.n, self.hx, self.hy, self.hz, self.dt, None)
        if self.mask is not None:
            s.mask = self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        return s

    def kernels(self):
        """[Mx | Kx | My | Ky | Mz | Kz], each of length 2n+1."""
        k = np.zeros(6 * (2 * self.n + 1))
        _check(lib().orc_problem_kernels(ctypes.byref(self._c()), _dp(k)))
        return k


def _check(rc):
    if rc < 0:
        raise RuntimeError(f"oracle returned {rc}")
    return rc


def bspline(n: int, x) -> np.ndarray:
    """Centred B-spline beta^n at x (Table tblBsplines, convolution row)."""
    L = lib()
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return np.array([L.orc_bspline(n, float(v)) for v in xs])


def bspline_deriv(n: int, x) -> np.ndarray:
    """beta^n' by the derivative identity of Table tblBsplines."""
    L = lib()
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return np.array([L.orc_bspline_deriv(n, float(v)) for v in xs])


def gauss_legendre(m: int):
    t = np.zeros(m)
    w = np.zeros(m)
    _check(lib().orc_gauss_legendre(m, _dp(t), _dp(w)))
    return t, w


def kernels_1d(n: int):
    """Unit-grid mass and stiffness kernels (2n+1 taps) by quadrature of their integrals."""
    m = np.zeros(2 * n + 1)
    k = np.zeros(2 * n + 1)
    _check(lib().orc_kernels_1d(n, _dp(m), _dp(k)))
    return m, k


def bspline_kernels(n: int, h: float):
    """Per-axis kernels M = h m, K = k / h."""
    M = np.zeros(2 * n + 1)
    K = np.zeros(2 * n + 1)
    _check(lib().orc_bspline_kernels(n, float(h), _dp(M), _dp(K)))
    return M, K


def _op(name, prob: Problem, x, kern=None):
    x = _f64(x).reshape(prob.shape)
    y = np.zeros(prob.shape)
    kern = prob.kernels() if kern is None else _f64(kern)
    _check(getattr(lib(), name)(ctypes.byref(prob._c()), _dp(kern), _dp(x), _dp(y)))
    return y


def op_stencil(prob: Problem, x, kern=None):
    """y = A x by the direct (2n+1)^3 stencil (Eq. tensForm, constant coefficients)."""
    return _op("orc_op_stencil", prob, x, kern)


def op_separable(prob: Problem, x, kern=None):
    """y = A x by the four separable 1-D convolution chains of Fig. FiltAlg."""
    return _op("orc_op_separable", prob, x, kern)


def op_points(prob: Problem, x, points, kern=None):
    """(A x) at the given flat indices only (direct stencil definition). x may be float32 or
    float64 (read as is, accumulated in double)."""
    x = np.ascontiguousarray(x)
    assert x.dtype in (np.float32, np.float64) and x.size == prob.nx * prob.ny * prob.nz
    pts = np.ascontiguousarray(points, dtype=np.int64)
    out = np.zeros(pts.size)
    kern = prob.kernels() if kern is None else _f64(kern)
    _check(lib().orc_op_points(ctypes.byref(prob._c()), _dp(kern), x.ctypes.data,
                               int(x.dtype == np.float32), pts.size,
                               pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _dp(out)))
    return out


def mass(prob: Problem, x, kern=None):
    """y = (Mz x My x Mx) x, the mass chain of Fig. FiltAlg alone."""
    return _op("orc_mass", prob, x, kern)


def bruteforce_matrix(prob: Problem, full3d: bool = False):
    """Dense Galerkin matrix over active nodes by Gauss quadrature of the basis (Eq.
    RitzGalerkin). Returns (A, active_flat_indices)."""
    L = lib()
    na = ctypes.c_int(0)
    _check(L.orc_bruteforce_matrix(ctypes.byref(prob._c()), int(full3d), None, ctypes.byref(na)))
    A = np.zeros((na.value, na.value))
    _check(L.orc_bruteforce_matrix(ctypes.byref(prob._c()), int(full3d), _dp(A), ctypes.byref(na)))
    if prob.mask is None:
        act = np.arange(prob.nx * prob.ny * prob.nz)
    else:
        act = np.flatnonzero(prob.mask.reshape(-1))
    return A, act


def dot(a, b) -> float:
    a = _f64(a).reshape(-1)
    b = _f64(b).reshape(-1)
    return lib().orc_dot(_dp(a), _dp(b), a.size)


def cg(prob: Problem, b, x0=None, tol=1e-10, max_iter=10000, kern=None):
    """Textbook CG (section 2.5). Returns (x, iterations, true relative residual, status)."""
    b = _f64(b).reshape(prob.shape)
    x = np.zeros(prob.shape) if x0 is None else _f64(x0).reshape(prob.shape).copy()
    kern = prob.kernels() if kern is None else _f64(kern)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _check(lib().orc_cg(ctypes.byref(prob._c()), _dp(kern), _dp(b), _dp(x), float(tol),
                             int(max_iter), ctypes.byref(it), ctypes.byref(rel)))
    return x, it.value, rel.value, st


def heat(prob: Problem, u0, q=None, nsteps=1, tol=1e-10, max_iter=10000, kern=None):
    """Implicit Euler steps (M + dt K) u^{k+1} = M (u^k + dt q). Returns (u, iters, relres, st)."""
    u = _f64(u0).reshape(prob.shape).copy()
    qq = None if q is None else _f64(q).reshape(prob.shape)
    kern = prob.kernels() if kern is None else _f64(kern)
    its = np.zeros(nsteps, dtype=np.int32)
    rel = np.zeros(nsteps)
    st = _check(lib().orc_heat(ctypes.byref(prob._c()), _dp(kern), _dp(u), _dp(qq), int(nsteps),
                               float(tol), int(max_iter),
                               its.ctypes.data_as(_I), _dp(rel)))
    return u, its, rel, st


def axis_rule(n: int, N: int, h: float):
    """Gauss rule on [0, (N+1)h] with n+1 points per half-cell (contains every knot)."""
    cap = 2 * (N + 1) * (n + 1)
    xs = np.zeros(cap)
    ws = np.zeros(cap)
    cnt = _check(lib().orc_axis_rule(n, N, float(h), _dp(xs), _dp(ws)))
    return xs[:cnt], ws[:cnt]


def eval_tensor(prob: Problem, c, xs, ys, zs):
    """u_h on the tensor grid zs x ys x xs (indirect B-spline transform, section 2.3)."""
    c = _f64(c).reshape(prob.shape)
    xs, ys, zs = _f64(xs), _f64(ys), _f64(zs)
    out = np.zeros((zs.size, ys.size, xs.size))
    _check(lib().orc_eval_tensor(ctypes.byref(prob._c()), 0, _dp(c), xs.size, _dp(xs), None,
                                 ys.size, _dp(ys), None, zs.size, _dp(zs), None, _dp(out)))
    return out


def load_tensor(prob: Problem, f, xs, wx, ys, wy, zs, wz):
    """l_i = sum_k w_k f(x_k) psi_i(x_k): load vector of f given on a weighted tensor grid."""
    f = _f64(f).reshape(len(zs), len(ys), len(xs))
    xs, wx, ys, wy, zs, wz = (_f64(v) for v in (xs, wx, ys, wy, zs, wz))
    out = np.zeros(prob.shape)
    _check(lib().orc_eval_tensor(ctypes.byref(prob._c()), 1, _dp(f), xs.size, _dp(xs), _dp(wx),
                                 ys.size, _dp(ys), _dp(wy), zs.size, _dp(zs), _dp(wz), _dp(out)))
    return out


def abs_op(prob: Problem, x):
    """(|A| |x|): the operator with every kernel tap and every ghost-extended coefficient
    replaced by its absolute value; the scale against which operator errors are measured
    (the stiffness kernel sums to zero)."""
    return _op("orc_abs_op", prob, x)


def set_plant(mode: int) -> None:
    """Test hook: 0 = correct odd reflection, 1 = zero ghosts, 2 = even reflection (solution),
    3 = zero ghosts for the coefficient fields of the variable-coefficient operator, 4 = the far
    face left out of the Robin boundary term."""
    lib().orc_set_plant(int(mode))


def sampled_basis_1d(n: int, N: int, h: float = None) -> np.ndarray:
    """B[j, i] = psi_i(x_j): the odd-reflected degree-n basis function of unknown i sampled at
    node j of an axis with N unknowns (positions (j + 1) h, faces at 0 and (N + 1) h). The
    reflected function is the B-spline centred at (i + 1) minus its mirror images about the
    faces (Eq. expansion with the zero-Dirichlet reading); in units of h it does not depend on h.
    This matrix is the indirect B-spline transform at the nodes along one axis (Fig.
    figBspnSignProc, section 2.3)."""
    P = 2 * (N + 1)                  # the odd extension is periodic with this period
    B = np.zeros((N, N))
    for i in range(N):
        I = i + 1
        for j in range(N):
            J = j + 1
            v = 0.0
            # images of the odd, P-periodic extension: +I + m P and -(I) + m P, m = -1, 0, 1
            for s, c in ((1.0, I), (1.0, I + P), (1.0, I - P), (-1.0, -I), (-1.0, -I + P),
                         (-1.0, -I - P)):
                if abs(J - c) < (n + 1) / 2.0:
                    v += s * float(lib().orc_bspline(n, float(J - c)))
            B[j, i] = v
    return B


def indirect_transform(prob: Problem, c) -> np.ndarray:
    """u at the grid nodes from the coefficients c (indirect B-spline transform, section 2.3):
    u = (Bz (x) By (x) Bx) c with the sampled reflected basis of each axis. The mask is not
    applied (the transform acts on the whole box)."""
    c = _f64(c).reshape(prob.shape)
    Bx = sampled_basis_1d(prob.n, prob.nx)
    By = sampled_basis_1d(prob.n, prob.ny)
    Bz = sampled_basis_1d(prob.n, prob.nz)
    return np.einsum("ck,bj,ai,kji->cba", Bz, By, Bx, c, optimize=True)


def direct_transform(prob: Problem, f) -> np.ndarray:
    """Coefficients c whose indirect transform reproduces the samples f at the nodes (direct
    B-spline transform by interpolation, section 2.3): one linear solve per axis with the
    sampled reflected basis, c = (Bz^-1 (x) By^-1 (x) Bx^-1) f."""
    f = _f64(f).reshape(prob.shape)
    Bx = sampled_basis_1d(prob.n, prob.nx)
    By = sampled_basis_1d(prob.n, prob.ny)
    Bz = sampled_basis_1d(prob.n, prob.nz)
    t = np.linalg.solve(Bx, f.reshape(-1, prob.nx).T).T.reshape(prob.shape)
    t = np.moveaxis(np.linalg.solve(By, np.moveaxis(t, 1, 0).reshape(prob.ny, -1)).reshape(
        prob.ny, prob.nz, prob.nx), 0, 1)
    t = np.linalg.solve(Bz, t.reshape(prob.nz, -1)).reshape(prob.shape)
    return t


# --- variable coefficients (Eq. RitzGalerkin / Eq. tensForm with D, mu_a in B-splines) -------

def coef_shape(prob: Problem):
    """Shape of a nodal coefficient field: the N + 2 nodes 0..N+1 of each axis, faces included
    (unknown i sits at node i + 1)."""
    return (prob.nz + 2, prob.ny + 2, prob.nx + 2)


def triple_kernels_1d(n: int):
    """(f1, w1), each (2n+1, 2n+1) indexed [a + n, b + n]: f1 = int beta(x) beta(x-a) beta(x-b),
    w1 = int beta'(x) beta'(x-a) beta(x-b), the per-axis factors of f^{klm} and w^{klm}
    (Eq. tensForm, section 2.4)."""
    L = 2 * n + 1
    f1 = np.zeros(L * L)
    w1 = np.zeros(L * L)
    _check(lib().orc_triple_kernels_1d(int(n), _dp(f1), _dp(w1)))
    return f1.reshape(L, L), w1.reshape(L, L)


def _var(name, prob: Problem, d, m, x):
    d = _f64(d).reshape(coef_shape(prob))
    m = _f64(m).reshape(coef_shape(prob))
    x = _f64(x).reshape(prob.shape)
    y = np.zeros(prob.shape)
    _check(getattr(lib(), name)(ctypes.byref(prob._c()), _dp(d), _dp(m), _dp(x), _dp(y)))
    return y


def op_var(prob: Problem, d, m, x):
    """y = A(d, m) x: the variable-coefficient operator sum_k sum_m x_k (dt d_m w^{klm} +
    m_m f^{klm}) of Eq. tensForm (no boundary term), written as the plain double sum over the
    solution and coefficient B-splines. d, m: nodal fields of shape coef_shape(prob), extended
    evenly across the faces; x odd-reflected and masked as for the constant operator."""
    return _var("orc_op_var", prob, d, m, x)


def abs_op_var(prob: Problem, d, m, x):
    """(|A(d, m)| |x|): every factor of every term replaced by its absolute value (error scale)."""
    return _var("orc_abs_op_var", prob, d, m, x)


def bruteforce_apply_var(prob: Problem, d, m, x):
    """A(d, m) x by Gauss quadrature over [0,1]^3 of dt D grad psi_i . grad u + mu_a psi_i u,
    every function evaluated pointwise (odd-reflected solution basis, even-reflected
    coefficient basis). Tiny grids only."""
    return _var("orc_bruteforce_apply_var", prob, d, m, x)


def op_var_points(prob: Problem, d, m, x, points, absolute=False):
    """(A(d, m) x) at the given flat indices only; x float32 or float64. absolute=True gives
    the (|A(d, m)| |x|) scale at those points instead."""
    d = _f64(d).reshape(coef_shape(prob))
    m = _f64(m).reshape(coef_shape(prob))
    x = np.ascontiguousarray(x)
    assert x.dtype in (np.float32, np.float64) and x.size == prob.nx * prob.ny * prob.nz
    pts = np.ascontiguousarray(points, dtype=np.int64)
    out = np.zeros(pts.size)
    _check(lib().orc_op_var_points(ctypes.byref(prob._c()), _dp(d), _dp(m), x.ctypes.data,
                                   int(x.dtype == np.float32), int(bool(absolute)), pts.size,
                                   pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _dp(out)))
    return out


# --- Robin (boundary penalty) problems on the box, Jacobi PCG, coarse-grid prolongation --------

def robin_size(n: int, N: int) -> int:
    """Unknowns per axis of the untruncated basis on a box of N interior nodes:
    N + 2 + 2 floor(n/2) (every B-spline whose support meets the box)."""
    return int(lib().orc_robin_size(int(n), int(N)))


def robin_shape(prob: Problem):
    return tuple(robin_size(prob.n, N) for N in (prob.nz, prob.ny, prob.nx))


def robin_1d(n: int, N: int, h: float):
    """(M, K, E): truncated Gram, stiffness and face matrices of one axis (dense Nt x Nt)."""
    Nt = robin_size(n, N)
    M, K, E = np.zeros(Nt * Nt), np.zeros(Nt * Nt), np.zeros(Nt * Nt)
    _check(lib().orc_robin_1d(int(n), int(N), float(h), _dp(M), _dp(K), _dp(E)))
    return M.reshape(Nt, Nt), K.reshape(Nt, Nt), E.reshape(Nt, Nt)


def _robin(name, prob: Problem, pen, x):
    x = _f64(x).reshape(robin_shape(prob))
    y = np.zeros(robin_shape(prob))
    _check(getattr(lib(), name)(ctypes.byref(prob._c()), float(pen), _dp(x), _dp(y)))
    return y


def op_robin(prob: Problem, pen, x):
    """A_R x: M + dt K + pen E over the untruncated basis, integrals truncated to the box (Eq.
    RitzGalerkin with the boundary term), x of shape robin_shape(prob)."""
    return _robin("orc_op_robin", prob, pen, x)


def abs_op_robin(prob: Problem, pen, x):
    return _robin("orc_abs_op_robin", prob, pen, x)


def bruteforce_apply_robin(prob: Problem, pen, x):
    """A_R x by volume and surface Gauss quadrature of point values of the basis (tiny grids)."""
    return _robin("orc_bruteforce_apply_robin", prob, pen, x)


def diag(prob: Problem, pen=0.0, robin=False):
    """Diagonal of the reflected (masked) operator, or of A_R with robin=True."""
    shape = robin_shape(prob) if robin else prob.shape
    d = np.zeros(shape)
    _check(lib().orc_diag(ctypes.byref(prob._c()), float(pen), int(bool(robin)), _dp(d)))
    return d


def pcg(prob: Problem, b, x0=None, tol=1e-10, max_iter=10000, pen=0.0, robin=False):
    """Jacobi-preconditioned CG. Returns (x, iterations, true relative residual, status)."""
    shape = robin_shape(prob) if robin else prob.shape
    b = _f64(b).reshape(shape)
    x = np.zeros(shape) if x0 is None else _f64(x0).reshape(shape).copy()
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _check(lib().orc_pcg(ctypes.byref(prob._c()), float(pen), int(bool(robin)), _dp(b), _dp(x),
                              float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rel)))
    return x, it.value, rel.value, st


def transfer_1d(n: int, Nf: int, hf: float, Nc: int, hc: float):
    T = np.zeros(robin_size(n, Nf) * robin_size(n, Nc))
    _check(lib().orc_transfer_1d(int(n), int(Nf), float(hf), int(Nc), float(hc), _dp(T)))
    return T.reshape(robin_size(n, Nf), robin_size(n, Nc))


def prolong_robin(fine: Problem, coarse: Problem, xc):
    """L2 projection of the coarse Robin expansion onto the fine Robin basis of the same box."""
    xc = _f64(xc).reshape(robin_shape(coarse))
    xf = np.zeros(robin_shape(fine))
    _check(lib().orc_prolong_robin(ctypes.byref(fine._c()), ctypes.byref(coarse._c()), _dp(xc), _dp(xf)))
    return xf


def diag_var(prob: Problem, d, m):
    """Diagonal of A(d, m) (inactive nodes: 1), each entry from the triple-sum definition."""
    d = _f64(d).reshape(coef_shape(prob))
    m = _f64(m).reshape(coef_shape(prob))
    out = np.zeros(prob.shape)
    _check(lib().orc_diag_var(ctypes.byref(prob._c()), _dp(d), _dp(m), _dp(out)))
    return out


def pcg_var(prob: Problem, d, m, b, x0=None, tol=1e-10, max_iter=10000):
    """Jacobi-preconditioned CG on A(d, m). Returns (x, iterations, true relative residual, status)."""
    d = _f64(d).reshape(coef_shape(prob))
    m = _f64(m).reshape(coef_shape(prob))
    b = _f64(b).reshape(prob.shape)
    x = np.zeros(prob.shape) if x0 is None else _f64(x0).reshape(prob.shape).copy()
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _check(lib().orc_pcg_var(ctypes.byref(prob._c()), _dp(d), _dp(m), _dp(b), _dp(x), float(tol),
                                  int(max_iter), ctypes.byref(it), ctypes.byref(rel)))
    return x, it.value, rel.value, st


def op_robin_points(prob: Problem, pen, x, points, absolute=False):
    """(A_R x) at the given flat indices of the Robin grid only; x float32 or float64;
    absolute=True gives the (|A_R| |x|) scale there."""
    x = np.ascontiguousarray(x)
    assert x.dtype in (np.float32, np.float64) and x.size == int(np.prod(robin_shape(prob)))
    pts = np.ascontiguousarray(points, dtype=np.int64)
    out = np.zeros(pts.size)
    _check(lib().orc_op_robin_points(ctypes.byref(prob._c()), float(pen), x.ctypes.data,
                                     int(x.dtype == np.float32), int(bool(absolute)), pts.size,
                                     pts.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _dp(out)))
    return out
