"""Pins of the variable-coefficient oracle (Eq. RitzGalerkin / Eq. tensForm of arXiv:1904.03057
with D(x) and mu_a(x) expanded in B-splines, section 2.3): closed-form triple products of the
linear B-spline, partition-of-unity reductions to the pinned two-product kernels, symmetries,
the constant-coefficient operator as the special case d = m = 1, a brute-force Galerkin
quadrature over the box with every function evaluated pointwise, and a planted boundary
mistake that the brute force catches."""
import numpy as np
import pytest

import oracle

DEGREES = [1, 2, 3, 4, 5]


def test_linear_triple_products_closed_form():
    """For the hat function beta^1, the integrals are elementary: int hat^3 = 1/2,
    int hat(x)^2 hat(x-1) = int_0^1 (1-x)^2 x = 1/12, int hat(x) hat(x-1)^2 = 1/12, and the
    supports of hat(x-1) and hat(x+1) meet in one point only. With hat' = +1 on (-1,0) and -1
    on (0,1): int hat'^2 hat = 1, int hat'^2 hat(x-1) = int_0^1 x = 1/2,
    int hat'(x) hat'(x-1) hat(x) = -int_0^1 (1-x) = -1/2, int hat'(x) hat'(x-1) hat(x-1) = -1/2."""
    f1, w1 = oracle.triple_kernels_1d(1)
    F = {(0, 0): 1 / 2, (0, 1): 1 / 12, (0, -1): 1 / 12, (1, 0): 1 / 12, (-1, 0): 1 / 12,
         (1, 1): 1 / 12, (-1, -1): 1 / 12, (1, -1): 0.0, (-1, 1): 0.0}
    W = {(0, 0): 1.0, (0, 1): 1 / 2, (0, -1): 1 / 2, (1, 0): -1 / 2, (-1, 0): -1 / 2,
         (1, 1): -1 / 2, (-1, -1): -1 / 2, (1, -1): 0.0, (-1, 1): 0.0}
    for (a, b), v in F.items():
        assert f1[a + 1, b + 1] == pytest.approx(v, abs=1e-15), (a, b)
    for (a, b), v in W.items():
        assert w1[a + 1, b + 1] == pytest.approx(v, abs=1e-15), (a, b)


@pytest.mark.parametrize("n", DEGREES)
def test_triple_products_reduce_to_kernels(n):
    """The integer shifts of beta^n sum to 1 (partition of unity), so summing the coefficient
    index b out of the triple products gives the two-product mass and stiffness kernels, which
    are pinned to exact rationals elsewhere."""
    f1, w1 = oracle.triple_kernels_1d(n)
    m1, k1 = oracle.kernels_1d(n)
    assert np.max(np.abs(f1.sum(axis=1) - m1)) <= 1e-15
    assert np.max(np.abs(w1.sum(axis=1) - k1)) <= 1e-14


@pytest.mark.parametrize("n", DEGREES)
def test_triple_product_symmetries(n):
    """f1(a, b) = f1(b, a) (the two non-derivative factors commute), f1(a, b) = f1(-a, -b)
    (beta^n is even), and the shift x -> x + a gives f1(a, b) = f1(-a, b - a) and
    w1(a, b) = w1(-a, b - a)."""
    f1, w1 = oracle.triple_kernels_1d(n)
    assert np.max(np.abs(f1 - f1.T)) <= 1e-15
    assert np.max(np.abs(f1 - f1[::-1, ::-1])) <= 1e-15
    assert np.max(np.abs(w1 - w1[::-1, ::-1])) <= 1e-15
    for a in range(-n, n + 1):
        for b in range(-n, n + 1):
            if abs(b - a) <= n:
                assert abs(f1[a + n, b + n] - f1[-a + n, b - a + n]) <= 1e-15
                assert abs(w1[a + n, b + n] - w1[-a + n, b - a + n]) <= 1e-15


def _case(n, dims, seed, masked=True, aniso=True):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    h = (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1)) if aniso else (1 / (nx + 1),) * 3
    mask = (rng.random((nz, ny, nx)) < 0.8).astype(np.uint8) if masked else None
    P = oracle.Problem(nx, ny, nz, n, *h, dt=0.03, mask=mask)
    d = rng.uniform(0.5, 2.0, oracle.coef_shape(P))
    m = rng.uniform(0.5, 2.0, oracle.coef_shape(P))
    x = rng.standard_normal(P.shape)
    return P, d, m, x, rng


@pytest.mark.parametrize("n", DEGREES)
def test_unit_coefficients_give_constant_operator(n):
    """d = m = 1 everywhere (ghosts included) makes D = mu_a = 1, so A(d, m) is the
    constant-coefficient operator M + dt K."""
    P, d, m, x, _ = _case(n, (6, 5, 7), 10 + n)
    one = np.ones(oracle.coef_shape(P))
    y = oracle.op_var(P, one, one, x)
    y0 = oracle.op_stencil(P, x)
    assert np.max(np.abs(y - y0)) <= 1e-13 * np.max(oracle.abs_op(P, x))


@pytest.mark.parametrize("n,dims", [(1, (4, 5, 3)), (2, (5, 4, 4)), (3, (5, 6, 4)),
                                    (4, (5, 5, 6)), (5, (6, 5, 5))])
def test_matches_bruteforce_quadrature(n, dims):
    """The triple-sum definition equals the Galerkin integral over the box computed from point
    values of the odd-reflected solution basis and the even-reflected coefficient basis."""
    P, d, m, x, _ = _case(n, dims, 20 + n)
    y = oracle.op_var(P, d, m, x)
    yb = oracle.bruteforce_apply_var(P, d, m, x)
    assert np.max(np.abs(y - yb)) <= 1e-12 * np.max(oracle.abs_op_var(P, d, m, x))


@pytest.mark.parametrize("n", [2, 3, 5])
def test_planted_zero_coefficient_ghosts_caught(n):
    """Zero instead of even-reflected coefficient ghosts changes D and mu_a near the faces;
    the brute-force quadrature (which never forms ghosts) sees the difference. (At n = 1 the
    operator reads no coefficient beyond the face nodes.)"""
    P, d, m, x, _ = _case(n, (5, 5, 5), 30 + n, masked=False)
    yb = oracle.bruteforce_apply_var(P, d, m, x)
    scale = np.max(oracle.abs_op_var(P, d, m, x))
    oracle.set_plant(3)
    try:
        yp = oracle.op_var(P, d, m, x)
    finally:
        oracle.set_plant(0)
    assert np.max(np.abs(yp - yb)) > 1e-3 * scale


@pytest.mark.parametrize("n", DEGREES)
def test_symmetric_and_linear_in_coefficients(n):
    """A(d, m) is symmetric on the active set, and linear in (d, m) at fixed x."""
    P, d, m, x, rng = _case(n, (6, 7, 5), 40 + n)
    mask = P.mask
    z = rng.standard_normal(P.shape) * mask
    xm = x * mask
    s1 = np.sum(z * oracle.op_var(P, d, m, xm))
    s2 = np.sum(xm * oracle.op_var(P, d, m, z))
    assert abs(s1 - s2) <= 1e-12 * np.sum(np.abs(z) * oracle.abs_op_var(P, d, m, xm))
    d2 = rng.uniform(-1, 1, d.shape)
    m2 = rng.uniform(-1, 1, m.shape)
    lhs = oracle.op_var(P, d + d2, m + m2, x)
    rhs = oracle.op_var(P, d, m, x) + oracle.op_var(P, d2, m2, x)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(oracle.abs_op_var(P, np.abs(d) + np.abs(d2),
                                                                          np.abs(m) + np.abs(m2), x))


def test_points_match_full():
    P, d, m, x, rng = _case(3, (9, 8, 7), 50)
    y = oracle.op_var(P, d, m, x)
    pts = rng.choice(x.size, 40, replace=False)
    assert np.array_equal(oracle.op_var_points(P, d, m, x, pts), y.reshape(-1)[pts])


@pytest.mark.parametrize("n,dims", [(1, (5, 4, 6)), (2, (5, 6, 4)), (3, (6, 5, 7))])
def test_diagonal_and_jacobi_pcg(n, dims):
    """The diagonal of A(d, m) (Jacobi preconditioner of the paper's large run) equals the
    diagonal of the dense matrix assembled column by column from the operator, reduces to the
    constant-coefficient diagonal at d = m = 1, and Jacobi PCG reaches the dense solution."""
    P, d, m, _, rng = _case(n, dims, 60 + n)
    d = rng.uniform(0.2, 5.0, d.shape)
    dg = oracle.diag_var(P, d, m)
    N = int(np.prod(P.shape))
    A = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        A[:, i] = oracle.op_var(P, d, m, e.reshape(P.shape)).reshape(-1)
    act = P.mask.reshape(-1).astype(bool)
    assert np.max(np.abs(np.diag(A)[act] - dg.reshape(-1)[act])) <= 1e-14 * np.max(np.abs(dg))
    one = np.ones(oracle.coef_shape(P))
    assert np.max(np.abs(oracle.diag_var(P, one, one) - oracle.diag(P))) <= 1e-14 * np.max(oracle.diag(P))
    b = rng.standard_normal(P.shape) * P.mask
    x, it, rel, st = oracle.pcg_var(P, d, m, b, tol=1e-11)
    xs = np.zeros(N)
    xs[act] = np.linalg.solve(A[np.ix_(act, act)], b.reshape(-1)[act])
    assert st == 0 and rel <= 1e-10
    assert np.max(np.abs(x.reshape(-1) - xs)) <= 1e-9 * np.max(np.abs(xs))
