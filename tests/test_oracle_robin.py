"""Pins of the Robin (boundary penalty) oracle: the untruncated B-spline basis on the box with
the boundary integral of Eq. RitzGalerkin, the Jacobi preconditioner of the paper's large run
and the coarse-grid prolongation (section 3). Closed forms from the cumulative B-spline,
brute-force volume and surface quadrature, the Dirichlet limit of a large penalty for linear
B-splines against the pinned reflected-basis solver, dense solves, exact prolongation between
nested grids, and a planted boundary mistake."""
import os
import numpy as np
import pytest

import oracle

DEGREES = [1, 2, 3, 4, 5]


def cum_bspline(n, t):
    """int_{-inf}^t beta^n(s) ds = sum_{k >= 0} beta^{n+1}(t - 1/2 - k): beta^{n+1} is the
    convolution of beta^n with the unit box, so its integer-shifted sum telescopes to the
    running integral."""
    kmax = max(0, int(np.ceil(t)) + n + 3)
    return sum(float(oracle.bspline(n + 1, np.array([t - 0.5 - k]))[0]) for k in range(kmax))


@pytest.mark.parametrize("n", DEGREES)
def test_one_dimensional_factors_closed_forms(n):
    """Row sums: M 1 = the integral of each B-spline over the box (cumulative B-spline), K 1 = 0
    (the B-splines sum to one on the box), E 1 = the face values; total E = 2 (two faces)."""
    N, h = 7, 1 / 8
    M, K, E = oracle.robin_1d(n, N, h)
    i0 = -(n // 2)
    for a in range(M.shape[0]):
        i = a + i0
        exact = h * (cum_bspline(n, (N + 1) - i) - cum_bspline(n, 0 - i))
        assert abs(M[a].sum() - exact) <= 1e-14
        face = float(oracle.bspline(n, np.array([0.0 - i]))[0] + oracle.bspline(n, np.array([N + 1.0 - i]))[0])
        assert abs(E[a].sum() - face) <= 1e-15
    assert np.max(np.abs(K.sum(axis=1))) <= 1e-12
    assert abs(E.sum() - 2.0) <= 1e-14 and abs(M.sum() - (N + 1) * h) <= 1e-14
    assert np.max(np.abs(M - M.T)) <= 1e-17 and np.linalg.eigvalsh(M).min() > 0
    # rows far from the faces are the shift-invariant kernels
    m1, k1 = oracle.bspline_kernels(n, h)
    mid = M.shape[0] // 2
    assert np.max(np.abs(M[mid, mid - n:mid + n + 1] - m1)) <= 1e-15
    assert np.max(np.abs(K[mid, mid - n:mid + n + 1] - k1)) <= 1e-12


@pytest.mark.parametrize("n,dims", [(1, (3, 4, 3)), (2, (3, 3, 4)), (3, (4, 3, 3)), (4, (4, 4, 5)),
                                    (5, (5, 5, 5))])
def test_matches_bruteforce_quadrature(n, dims):
    nx, ny, nz = dims
    P = oracle.Problem(nx, ny, nz, n, 1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1), dt=0.02)
    x = np.random.default_rng(n).standard_normal(oracle.robin_shape(P))
    y = oracle.op_robin(P, 3.7, x)
    yb = oracle.bruteforce_apply_robin(P, 3.7, x)
    assert np.max(np.abs(y - yb)) <= 1e-13 * np.max(oracle.abs_op_robin(P, 3.7, x))


def test_planted_missing_face_caught():
    P = oracle.Problem(4, 3, 3, 3, 1 / 5, 1 / 4, 1 / 4, dt=0.02)
    x = np.random.default_rng(9).standard_normal(oracle.robin_shape(P))
    yb = oracle.bruteforce_apply_robin(P, 3.7, x)
    oracle.set_plant(4)
    try:
        yp = oracle.op_robin(P, 3.7, x)
    finally:
        oracle.set_plant(0)
    assert np.max(np.abs(yp - yb)) > 1e-3 * np.max(oracle.abs_op_robin(P, 3.7, x))


def test_unit_coefficients_closed_form():
    """u = 1 (every coefficient 1): the stiffness term vanishes, the mass term is the product
    of the per-axis B-spline integrals and the penalty term adds the face values."""
    n, (nx, ny, nz) = 3, (5, 4, 6)
    hs = (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1))
    P = oracle.Problem(nx, ny, nz, n, *hs, dt=0.3)
    one = np.ones(oracle.robin_shape(P))
    y = oracle.op_robin(P, 2.0, one)
    i0 = -(n // 2)
    ints, faces = [], []
    for N, h in zip((nx, ny, nz), hs):
        Nt = oracle.robin_size(n, N)
        ints.append(np.array([h * (cum_bspline(n, N + 1 - (a + i0)) - cum_bspline(n, -(a + i0))) for a in range(Nt)]))
        faces.append(np.array([float(oracle.bspline(n, np.array([-(a + i0) + 0.0]))[0] +
                                     oracle.bspline(n, np.array([N + 1.0 - (a + i0)]))[0]) for a in range(Nt)]))
    Ix, Iy, Iz = ints
    Fx, Fy, Fz = faces
    ref = (np.einsum("k,j,i->kji", Iz, Iy, Ix) +
           2.0 * (np.einsum("k,j,i->kji", Fz, Iy, Ix) + np.einsum("k,j,i->kji", Iz, Fy, Ix) +
                  np.einsum("k,j,i->kji", Iz, Iy, Fx)))
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_large_penalty_tends_to_dirichlet_linear():
    """Linear B-splines: the interior hats vanish on the faces, so the reflected basis is the
    interior hats and a penalty p forces the face coefficients to O(1/p): the Robin solution
    tends to the Dirichlet solution of the pinned reflected-basis oracle, error O(1/p)."""
    n, N, dt = 1, 6, 0.01
    h = 1 / (N + 1)
    P = oracle.Problem(N, N, N, n, h, dt=dt)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(P.shape)
    xd, _, rel, st = oracle.cg(P, f, tol=1e-13)
    assert st == 0
    errs = []
    for pen in (1e3, 1e5):
        b = np.zeros(oracle.robin_shape(P))
        b[1:-1, 1:-1, 1:-1] = f            # the interior hats carry the same load
        xr, _, relr, str_ = oracle.pcg(P, b, tol=1e-13, pen=pen, robin=True, max_iter=20000)
        assert str_ == 0
        errs.append(np.max(np.abs(xr[1:-1, 1:-1, 1:-1] - xd)) / np.max(np.abs(xd)))
        assert np.max(np.abs(xr[0])) <= 10.0 / pen * np.max(np.abs(xd)) / h
    assert errs[1] < errs[0] / 30 and errs[1] < 1e-3


@pytest.mark.parametrize("robin", [False, True])
def test_jacobi_pcg_matches_dense_solve(robin):
    rng = np.random.default_rng(5)
    if robin:
        P = oracle.Problem(4, 5, 3, 2, 1 / 5, 1 / 6, 1 / 4, dt=0.01)
        shape = oracle.robin_shape(P)
        apply = lambda v: oracle.op_robin(P, 4.0, v)
    else:
        P = oracle.Problem(6, 5, 7, 3, 1 / 7, 1 / 6, 1 / 8, dt=0.01,
                           mask=(rng.random((7, 5, 6)) < 0.8).astype(np.uint8))
        shape = P.shape
        apply = lambda v: oracle.op_stencil(P, v)
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = apply(e.reshape(shape)).reshape(-1)
    d = oracle.diag(P, 4.0, robin=robin).reshape(-1)
    act = np.ones(n, bool) if robin else P.mask.reshape(-1).astype(bool)
    assert np.max(np.abs(np.diag(A)[act] - d[act])) <= 1e-14 * np.max(np.abs(d))
    b = rng.standard_normal(shape) * (1 if robin else P.mask)
    x, it, rel, st = oracle.pcg(P, b, tol=1e-12, pen=4.0, robin=robin, max_iter=5000)
    # the recursive residual reaches 1e-12; the true one trails it by the conditioning
    # (about 1e7 for the untruncated quadratic basis)
    assert st == 0 and rel <= 1e-9
    xs = np.zeros(n)
    xs[act] = np.linalg.solve(A[np.ix_(act, act)], b.reshape(-1)[act])
    assert np.max(np.abs(x.reshape(-1) - xs)) <= 1e-8 * np.max(np.abs(xs))


def _eval_robin(n, Ns, hs, c, pts):
    """u(p) = sum_i c_i beta(p/h - i) of a Robin expansion at points (x, y, z)."""
    i0 = -(n // 2)
    vals = []
    for p in pts:
        w = []
        for d in range(3):
            Nt = oracle.robin_size(n, Ns[d])
            w.append(oracle.bspline(n, p[d] / hs[d] - (np.arange(Nt) + i0)))
        vals.append(np.einsum("k,j,i,kji->", w[2], w[1], w[0], c))
    return np.array(vals)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_prolongation_exact_on_nested_grids(n):
    """Coarse step 2 h (N_c + 1 divides N_f + 1): the coarse spline space is contained in the
    fine one (for odd n the knots nest; for even n too, as the half-integer knots of the coarse
    grid are fine knots), so the L2 projection reproduces the coarse function exactly."""
    Nc, Nf = (3, 3, 4), (7, 7, 9)
    hc = tuple(1 / (N + 1) for N in Nc)
    hf = tuple(1 / (N + 1) for N in Nf)
    C = oracle.Problem(*Nc, n, *hc, dt=0.0)
    F = oracle.Problem(*Nf, n, *hf, dt=0.0)
    rng = np.random.default_rng(n)
    xc = rng.standard_normal(oracle.robin_shape(C))
    xf = oracle.prolong_robin(F, C, xc)
    pts = rng.uniform(0, 1, size=(40, 3))
    uc = _eval_robin(n, Nc, hc, xc, pts)
    uf = _eval_robin(n, Nf, hf, xf, pts)
    if n % 2 == 1:
        assert np.max(np.abs(uf - uc)) <= 1e-11 * np.max(np.abs(uc))
    # constants map to constants on any pair of grids (partition of unity)
    one = oracle.prolong_robin(F, C, np.ones(oracle.robin_shape(C)))
    assert np.max(np.abs(one - 1.0)) <= 1e-10


def test_points_match_full():
    P = oracle.Problem(6, 5, 7, 2, 1 / 7, 1 / 6, 1 / 8, dt=0.02)
    x = np.random.default_rng(11).standard_normal(oracle.robin_shape(P))
    y = oracle.op_robin(P, 4.5, x)
    pts = np.random.default_rng(12).choice(x.size, 50, replace=False)
    assert np.array_equal(oracle.op_robin_points(P, 4.5, x, pts), y.reshape(-1)[pts])
    assert np.array_equal(oracle.op_robin_points(P, 4.5, x, pts, absolute=True),
                          oracle.abs_op_robin(P, 4.5, x).reshape(-1)[pts])


def _flop1d_table():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "flop1d_bspline.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows[float(v[0])] = [int(c) for c in v[1:]]
    return rows


def _band_nonzeros(Nt, n):
    """Entries of an Nt x Nt matrix with half-bandwidth n."""
    return Nt * (2 * n + 1) - n * (n + 1)


def test_operation_counts_of_table_tblFlop1d():
    """The paper's operation counts for its 1-D Robin example on [-25, 25] (Table tblFlop1d,
    B-spline columns) are those of one product with the 1-D system matrix, nnz multiplies and
    nnz - Nt additions, over the untruncated basis. The oracle's matrices reproduce every printed
    count: for h = 1 and 0.5 by counting their nonzero entries (which also shows the band is full
    and nothing lies outside it), for all four steps through the basis size N + 2 + 2 floor(n/2)
    with the full band. A basis of N + n + 1 functions, or one without the outermost B-splines,
    misses the table."""
    table = _flop1d_table()
    assert sorted(table) == [0.125, 0.25, 0.5, 1.0]
    for h, counts in table.items():
        N = int(round(50 / h)) - 1          # interior nodes of [-25, 25] at step h
        for n, printed in zip(DEGREES, counts):
            Nt = oracle.robin_size(n, N)
            assert 2 * _band_nonzeros(Nt, n) - Nt == printed, (h, n)
            if h >= 0.5:
                M, K, E = oracle.robin_1d(n, N, h)
                A = K + M + 0.5 * E
                nnz = int(np.count_nonzero(A))
                assert nnz == _band_nonzeros(Nt, n), (h, n)
                assert np.count_nonzero(np.triu(A, n + 1)) == 0
                assert 2 * nnz - Nt == printed, (h, n)


def _robin_line_solution(x):
    """Closed-form solution of -phi'' + phi = exp(-(x/2)^2) on [-25, 25] with 2 phi'.n + phi = 0:
    the whole-line solution (the source convolved with exp(-|x|)/2, in erfc form) plus the even
    homogeneous term A cosh(x) that meets the end condition."""
    from scipy.special import erfc

    c = np.e * np.sqrt(np.pi) / 2

    def part(t):
        return c * (np.exp(-t) * erfc((2 - t) / 2) + np.exp(t) * erfc((t + 2) / 2))

    def dpart(t):
        return c * (-np.exp(-t) * erfc((2 - t) / 2) + np.exp(t) * erfc((t + 2) / 2))

    A = -(2 * dpart(25.0) + part(25.0)) / (2 * np.sinh(25.0) + np.cosh(25.0))
    return part(x) + A * np.cosh(x)


def test_one_dimensional_robin_example_converges_at_order_n_plus_1():
    """The paper's 1-D example (section 3: -(D phi')' + mu_a phi = exp(-(x/2)^2) on [-25, 25],
    2 D phi'.n + phi = 0, h = 2^-mu), with D = mu_a = 1 (the paper gives no values): the Galerkin
    system K + M + E/2 of the oracle's 1-D Robin matrices, solved densely, approaches the closed-form
    solution in L2 at order h^(n+1) for n = 1..5. A wrong scale of K or M, a dropped or shifted
    entry, or a wrong basis position breaks the rate."""
    g, w = np.polynomial.legendre.leggauss(8)
    for n in DEGREES:
        errs = []
        for h in (1.0, 0.5, 0.25):
            N = int(round(50 / h)) - 1
            M, K, E = oracle.robin_1d(n, N, h)
            Nt, i0 = M.shape[0], -(n // 2)
            t = (np.arange(N + 1)[:, None] + (g[None, :] + 1) / 2).ravel()   # node units
            wt = np.tile(w * h / 2, N + 1)
            xs = -25.0 + h * t
            # B[p, a] = beta^n(t_p - (a + i0)), only the n + 1 B-splines nonzero at t_p
            B = np.zeros((t.size, Nt))
            first = np.floor(t - (n + 1) / 2).astype(int) + 1 - i0
            for k in range(n + 1):
                a = first + k
                ok = (a >= 0) & (a < Nt)
                B[np.nonzero(ok)[0], a[ok]] = oracle.bspline(n, t[ok] - (a[ok] + i0))
            assert np.max(np.abs(B.sum(axis=1) - 1.0)) <= 1e-13   # every nonzero B-spline taken
            c = np.linalg.solve(K + M + 0.5 * E, B.T @ (wt * np.exp(-(xs / 2) ** 2)))
            errs.append(np.sqrt(np.sum(wt * (B @ c - _robin_line_solution(xs)) ** 2)))
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert n + 1 - 0.1 <= rates[-1] <= n + 2, (n, errs, rates)
