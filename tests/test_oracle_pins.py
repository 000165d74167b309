"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by itself.

Each pin is chosen so that a plausible mistake (a dropped term, a wrong sign or index, a
transposed operand, a wrong ghost rule) fails at least one of them; the planted-mistake tests at
the end check exactly that, by feeding the oracle wrong kernels or switching its ghost rule.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1904_03057_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# Independent exact B-spline (truncated-power form) in rational arithmetic
# ---------------------------------------------------------------------------------------------

def beta_exact(n: int, x: Fraction) -> Fraction:
    """Centred B-spline via the truncated-power sum (the (n+1)-fold convolution of the unit box,
    Table tblBsplines), evaluated exactly."""
    s = Fraction(0)
    half = Fraction(n + 1, 2)
    for k in range(n + 2):
        t = x + half - k
        if t > 0:
            s += (-1) ** k * math.comb(n + 1, k) * t ** n
    return s / math.factorial(n)


def exact_kernels(n: int):
    """m_j = beta^{2n+1}(j); k_j = -(beta^{2n-1}(j+1) - 2 beta^{2n-1}(j) + beta^{2n-1}(j-1))
    (scalar-product and derivative identities of Table tblBsplines)."""
    m = [beta_exact(2 * n + 1, Fraction(j)) for j in range(-n, n + 1)]
    k = [-(beta_exact(2 * n - 1, Fraction(j + 1)) - 2 * beta_exact(2 * n - 1, Fraction(j))
           + beta_exact(2 * n - 1, Fraction(j - 1))) for j in range(-n, n + 1)]
    return m, k


def symbol(taps, theta):
    """t^(theta) = sum_j t_j cos(j theta) for a symmetric kernel given on j = -n..n."""
    n = (len(taps) - 1) // 2
    return sum(float(t) * math.cos((j - n) * theta) for j, t in enumerate(taps))


# ---------------------------------------------------------------------------------------------
# B-spline values and kernels
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5])
def test_bspline_matches_exact_truncated_power(orc, n):
    pts = [Fraction(p, 7) for p in range(-28, 29)]
    got = orc.bspline(n, [float(p) for p in pts])
    want = np.array([float(beta_exact(n, p)) for p in pts])
    assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_bspline_partition_of_unity_and_derivative(orc, n):
    rng = np.random.default_rng(n)
    xs = rng.uniform(-0.5, 0.5, 20)
    for x in xs:
        s = sum(orc.bspline(n, x - k)[0] for k in range(-n - 2, n + 3))
        assert abs(s - 1.0) < 1e-14
    # derivative identity vs a central difference of the value
    for x in rng.uniform(-(n + 1) / 2, (n + 1) / 2, 20):
        e = 1e-6
        fd = (orc.bspline(n, x + e)[0] - orc.bspline(n, x - e)[0]) / (2 * e)
        assert abs(fd - orc.bspline_deriv(n, x)[0]) < 1e-7


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_kernels_equal_exact_rationals(orc, n):
    m, k = orc.kernels_1d(n)
    me, ke = exact_kernels(n)
    assert np.max(np.abs(m - np.array([float(v) for v in me]))) < 2e-16 * 8
    assert np.max(np.abs(k - np.array([float(v) for v in ke]))) < 2e-15
    # mass sums to one (partition of unity), stiffness to zero (constants have no energy)
    assert sum(me) == 1 and sum(ke) == 0
    assert abs(m.sum() - 1) < 1e-15 and abs(k.sum()) < 1e-14
    assert np.allclose(m, m[::-1], rtol=0, atol=0) and np.allclose(k, k[::-1], rtol=0, atol=0)


def test_cubic_kernels_golden(orc):
    rows = {}
    for line in open(os.path.join(GOLDEN, "cubic_kernels.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rows[key] = [int(v) for v in vals]
    m, k = orc.kernels_1d(3)
    assert np.allclose(m * rows["mass_denominator"][0], rows["mass_numerators"], atol=1e-11)
    assert np.allclose(k * rows["stiffness_denominator"][0], rows["stiffness_numerators"],
                       atol=1e-12)
    me, ke = exact_kernels(3)
    assert [v * 5040 for v in me] == rows["mass_numerators"]
    assert [v * 120 for v in ke] == rows["stiffness_numerators"]


def test_known_low_degree_tables():
    # n = 1: hat functions, the linear FEM matrices [1,4,1]/6 and [-1,2,-1]
    m, k = exact_kernels(1)
    assert m == [Fraction(1, 6), Fraction(4, 6), Fraction(1, 6)]
    assert k == [-1, 2, -1]
    m, k = exact_kernels(2)
    assert [v * 120 for v in m] == [1, 26, 66, 26, 1]
    assert [v * 6 for v in k] == [-1, -2, 6, -2, -1]


def test_scaled_kernels(orc):
    h = 1.0 / 37
    M, K = orc.bspline_kernels(3, h)
    m, k = orc.kernels_1d(3)
    assert np.allclose(M, h * m, rtol=1e-15) and np.allclose(K, k / h, rtol=1e-15)


# ---------------------------------------------------------------------------------------------
# Operator: brute-force Galerkin matrix, separable vs stencil, symmetry, closed forms
# ---------------------------------------------------------------------------------------------

def _rand_mask(shape, seed, frac=0.7):
    return (np.random.default_rng(seed).random(shape) < frac).astype(np.uint8)


CASES = [
    # (nx, ny, nz, n, dt, masked)
    (4, 4, 4, 1, 0.3, False),
    (5, 4, 6, 2, 0.05, True),
    (4, 5, 4, 3, 1.0, False),
    (6, 5, 4, 3, 0.01, True),
    (5, 5, 5, 4, 0.2, False),
    (5, 6, 5, 5, 0.02, True),
]


@pytest.mark.parametrize("nx,ny,nz,n,dt,masked", CASES)
def test_operator_equals_bruteforce_galerkin_matrix(orc, nx, ny, nz, n, dt, masked):
    mask = _rand_mask((nz, ny, nx), nx + 10 * n) if masked else None
    p = orc.Problem(nx, ny, nz, n, 1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1), dt=dt, mask=mask)
    A, act = orc.bruteforce_matrix(p)
    x = np.random.default_rng(7).standard_normal(p.shape)
    if mask is not None:
        x *= mask
    want = np.zeros(x.size)
    want[act] = A @ x.reshape(-1)[act]
    scale = np.max(np.abs(want))
    for y in (orc.op_stencil(p, x), orc.op_separable(p, x)):
        assert np.max(np.abs(y.reshape(-1) - want)) < 1e-13 * scale


@pytest.mark.parametrize("nx,ny,nz,n", [(3, 4, 3, 2), (4, 3, 4, 3)])
def test_bruteforce_full3d_equals_factorised(orc, nx, ny, nz, n):
    mask = _rand_mask((nz, ny, nx), 3)
    p = orc.Problem(nx, ny, nz, n, 1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1), dt=0.1, mask=mask)
    A1, _ = orc.bruteforce_matrix(p, full3d=False)
    A3, _ = orc.bruteforce_matrix(p, full3d=True)
    assert np.max(np.abs(A1 - A3)) < 1e-13 * np.max(np.abs(A1))


def test_operator_symmetric_positive_definite(orc):
    mask = inputs.sphere_mask(12, 11, 10, radius=0.4).numpy()
    p = orc.Problem(12, 11, 10, 3, 1 / 13, 1 / 12, 1 / 11, dt=2e-3, mask=mask)
    rng = np.random.default_rng(11)
    for _ in range(3):
        x = rng.standard_normal(p.shape) * mask
        y = rng.standard_normal(p.shape) * mask
        ax, ay = orc.op_separable(p, x), orc.op_separable(p, y)
        assert abs(np.vdot(x, ay) - np.vdot(ax, y)) < 1e-13 * np.linalg.norm(ax) * np.linalg.norm(y)
        assert np.vdot(x, ax) > 0


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_sine_modes_are_eigenvectors(orc, n):
    """c_i = prod_d sin(pi k_d i h_d) satisfies A c = lambda c, lambda from the cosine symbols
    of the exact rational kernels (odd reflection makes the sine modes exact eigenvectors)."""
    nx, ny, nz = 9, 10, 11
    hs = (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1))
    dt = 3e-3
    p = orc.Problem(nx, ny, nz, n, *hs, dt=dt)
    me, ke = exact_kernels(n)
    for kv in [(1, 1, 1), (2, 5, 3), (9, 1, 11)]:
        c = inputs.sine_mode_field(nx, ny, nz, [(kv, 1.0)]).numpy()
        th = [math.pi * kv[d] * hs[d] for d in range(3)]
        mh = [hs[d] * symbol(me, th[d]) for d in range(3)]
        kh = [symbol(ke, th[d]) / hs[d] for d in range(3)]
        lam = mh[0] * mh[1] * mh[2] + dt * (kh[0] * mh[1] * mh[2] + mh[0] * kh[1] * mh[2]
                                            + mh[0] * mh[1] * kh[2])
        y = orc.op_separable(p, c)
        assert np.max(np.abs(y - lam * c)) < 1e-13 * np.max(np.abs(lam * c)) + 1e-18
        ys = orc.op_stencil(p, c)
        assert np.max(np.abs(ys - lam * c)) < 1e-13 * np.max(np.abs(lam * c)) + 1e-18


def test_constant_field_interior(orc):
    """Away from the faces, the mass operator maps a constant to h^3 times it (mass kernel sums
    to one) and each stiffness chain maps it to zero (stiffness kernel sums to zero)."""
    N, n = 20, 3
    h = 1 / (N + 1)
    p = orc.Problem(N, N, N, n, h, dt=0.7)
    c = np.full(p.shape, 2.5)
    y = orc.op_separable(p, c)
    inner = y[n:-n, n:-n, n:-n]
    assert np.max(np.abs(inner - 2.5 * h ** 3)) < 1e-15 * 2.5 / h


# ---------------------------------------------------------------------------------------------
# Solver pins
# ---------------------------------------------------------------------------------------------

def test_cg_solves_against_dense_solve(orc):
    mask = _rand_mask((5, 6, 7), 9, 0.8)
    p = orc.Problem(7, 6, 5, 3, 1 / 8, 1 / 7, 1 / 6, dt=0.02, mask=mask)
    A, act = orc.bruteforce_matrix(p)
    b = np.random.default_rng(5).standard_normal(p.shape) * mask
    x, it, rel, st = orc.cg(p, b, tol=1e-13, max_iter=500)
    want = np.linalg.solve(A, b.reshape(-1)[act])
    assert st == 0 and rel < 1e-12
    assert np.max(np.abs(x.reshape(-1)[act] - want)) < 1e-9 * np.max(np.abs(want))
    assert np.all(x.reshape(-1)[np.setdiff1d(np.arange(x.size), act)] == 0)


def test_cg_one_iteration_for_eigenvector(orc):
    N = 16
    p = orc.Problem(N, N, N, 3, 1 / (N + 1), dt=1e-3)
    b = inputs.sine_mode_field(N, N, N, [((1, 1, 1), 1.0)]).numpy()
    x, it, rel, st = orc.cg(p, b, tol=1e-10)
    assert st == 0 and it == 1 and rel < 1e-12


def test_heat_sine_mode_decay_closed_form(orc):
    """Config-1 shape at N = 16: u^{K} = g^K u^0 with g = (prod h m^) / lambda."""
    N, n, dt, K = 16, 3, 1e-3, 10
    h = 1 / (N + 1)
    p = orc.Problem(N, N, N, n, h, dt=dt)
    u0 = inputs.sine_mode_field(N, N, N, [((1, 1, 1), 1.0)]).numpy()
    u, its, rel, st = orc.heat(p, u0, None, K, tol=1e-12)
    me, ke = exact_kernels(n)
    th = math.pi * h
    mh, kh = h * symbol(me, th), symbol(ke, th) / h
    lam = mh ** 3 + dt * 3 * kh * mh ** 2
    g = mh ** 3 / lam
    assert st == 0
    assert np.max(np.abs(u - g ** K * u0)) < 1e-11
    # and the discrete decay factor approaches the implicit-Euler factor 1/(1 + 3 pi^2 dt)
    assert abs(g - 1 / (1 + 3 * math.pi ** 2 * dt)) < 1e-6


def test_heat_source_rhs_is_mass_of_u_plus_dt_q(orc):
    """With u0 = 0 and a source q that is one sine mode, one step gives u = dt g q."""
    N, n, dt = 12, 2, 2e-3
    h = 1 / (N + 1)
    p = orc.Problem(N, N, N, n, h, dt=dt)
    q = inputs.sine_mode_field(N, N, N, [((2, 1, 3), 1.0)]).numpy()
    u, its, rel, st = orc.heat(p, np.zeros(p.shape), q, 1, tol=1e-13)
    me, ke = exact_kernels(n)
    mh = [h * symbol(me, math.pi * k * h) for k in (2, 1, 3)]
    kh = [symbol(ke, math.pi * k * h) / h for k in (2, 1, 3)]
    M3 = mh[0] * mh[1] * mh[2]
    lam = M3 + dt * (kh[0] * mh[1] * mh[2] + mh[0] * kh[1] * mh[2] + mh[0] * mh[1] * kh[2])
    assert np.max(np.abs(u - dt * M3 / lam * q)) < 1e-12 * np.max(np.abs(q))


@pytest.mark.parametrize("n", [2, 3])
def test_spatial_convergence_order(orc, n):
    """One implicit Euler step from u0 = sin sin sin: the Galerkin solution converges in L2 to
    the time-discrete exact solution u0 / (1 + 3 pi^2 dt) at order h^{n+1}."""
    dt = 1e-3
    errs, hs = [], []
    for N in (7, 15, 31):
        h = 1 / (N + 1)
        p = orc.Problem(N, N, N, n, h, dt=dt)
        xs, ws = orc.axis_rule(n, N, h)
        s = np.sin(np.pi * xs)
        f = s[:, None, None] * s[None, :, None] * s[None, None, :]
        load = orc.load_tensor(p, f, xs, ws, xs, ws, xs, ws)
        c, it, rel, st = orc.cg(p, load, tol=1e-14, max_iter=2000)
        uh = orc.eval_tensor(p, c, xs, xs, xs)
        ex = f / (1 + 3 * np.pi ** 2 * dt)
        w3 = ws[:, None, None] * ws[None, :, None] * ws[None, None, :]
        errs.append(math.sqrt(float(np.sum(w3 * (uh - ex) ** 2))))
        hs.append(h)
    rate = math.log(errs[-2] / errs[-1]) / math.log(hs[-2] / hs[-1])
    assert rate > n + 1 - 0.35, (errs, rate)


# ---------------------------------------------------------------------------------------------
# Planted mistakes: each must fail a pin above
# ---------------------------------------------------------------------------------------------

def _bruteforce_gap(orc, p, kern=None):
    A, act = orc.bruteforce_matrix(p)
    x = np.random.default_rng(1).standard_normal(p.shape)
    if p.mask is not None:
        x *= p.mask
    want = np.zeros(x.size)
    want[act] = A @ x.reshape(-1)[act]
    y = orc.op_separable(p, x, kern)
    return np.max(np.abs(y.reshape(-1) - want)) / np.max(np.abs(want))


def test_planted_kernel_mistakes_are_caught(orc):
    p = orc.Problem(5, 6, 7, 3, 1 / 6, 1 / 7, 1 / 8, dt=0.05)
    good = p.kernels()
    assert _bruteforce_gap(orc, p, good) < 1e-13
    L = 7
    planted = []
    k = good.copy(); k[L + 2] = -k[L + 2]; planted.append(k)          # sign of one stiffness tap
    k = good.copy(); k[0] = 0.0; planted.append(k)                     # dropped mass tap
    k = good.copy(); k[0:2 * L], k[2 * L:4 * L] = good[2 * L:4 * L].copy(), good[0:2 * L].copy()
    planted.append(k)                                                  # x and y kernels swapped
    k = good.copy(); k[L:2 * L] = np.roll(good[L:2 * L], 1); planted.append(k)  # shifted index
    for k in planted:
        assert _bruteforce_gap(orc, p, k) > 1e-6


def test_planted_ghost_rule_mistakes_are_caught(orc):
    p = orc.Problem(6, 5, 6, 3, 1 / 7, 1 / 6, 1 / 7, dt=0.05)
    try:
        for mode in (1, 2):
            orc.set_plant(mode)
            assert _bruteforce_gap(orc, p) > 1e-6
    finally:
        orc.set_plant(0)
    assert _bruteforce_gap(orc, p) < 1e-13


# ---- B-spline transforms at the nodes (section 2.3, Fig. figBspnSignProc) -----------------------

def test_indirect_transform_matches_independent_evaluator():
    """The sampled-basis transform equals the oracle's point evaluator (psi_1d in C) at the
    nodes, for every degree and anisotropic steps."""
    rng = np.random.default_rng(31)
    for n in range(1, 6):
        p = oracle.Problem(9, 7, 8, n, 1 / 10, hy=1 / 8, hz=1 / 9)
        c = rng.standard_normal(p.shape)
        xs = (np.arange(p.nx) + 1) * p.hx
        ys = (np.arange(p.ny) + 1) * p.hy
        zs = (np.arange(p.nz) + 1) * p.hz
        assert np.max(np.abs(oracle.eval_tensor(p, c, xs, ys, zs) - oracle.indirect_transform(p, c))) <= 1e-13


def test_direct_transform_sine_closed_form():
    """Sine modes are eigenvectors of the sampled odd-reflected basis: the direct transform of
    prod_d sin(pi k_d x_d) is the same field divided by prod_d sum_j beta^n(j) cos(pi k_d j h_d)."""
    for n in (1, 2, 3, 4, 5):
        N = (11, 9, 10)
        p = oracle.Problem(N[0], N[1], N[2], n, 1 / (N[0] + 1), hy=1 / (N[1] + 1), hz=1 / (N[2] + 1))
        k = (3, 2, 5)
        hs = (p.hx, p.hy, p.hz)
        axes = [np.sin(np.pi * k[d] * (np.arange(N[d]) + 1) * hs[d]) for d in range(3)]
        f = axes[2][:, None, None] * axes[1][None, :, None] * axes[0][None, None, :]
        lam = 1.0
        for d in range(3):
            js = np.arange(-3, 4)
            lam *= float(np.sum(oracle.bspline(n, js) * np.cos(np.pi * k[d] * js * hs[d])))
        c = oracle.direct_transform(p, f)
        assert np.max(np.abs(c - f / lam)) <= 1e-12 * np.max(np.abs(f / lam)), n


def test_direct_transform_degree_one_is_identity_and_round_trip():
    rng = np.random.default_rng(32)
    p1 = oracle.Problem(6, 5, 7, 1, 1 / 7)
    f = rng.standard_normal(p1.shape)
    assert np.max(np.abs(oracle.direct_transform(p1, f) - f)) <= 1e-15
    p3 = oracle.Problem(12, 10, 11, 3, 1 / 13)
    f = rng.standard_normal(p3.shape)
    assert np.max(np.abs(oracle.indirect_transform(p3, oracle.direct_transform(p3, f)) - f)) <= 1e-12


def test_planted_missing_reflection_in_transform_is_caught():
    """A sampled basis without the mirror images (no zero-Dirichlet reflection) differs at the
    nodes next to the faces, and the closed form catches it (degree 5, whose samples reach two
    nodes: the cubic's vanish one node beyond the face)."""
    n, N = 5, 10
    B = oracle.sampled_basis_1d(n, N)
    Bbad = np.array([[float(oracle.bspline(n, (j + 1) - (i + 1))[0]) for i in range(N)] for j in range(N)])
    k, h = 2, 1 / (N + 1)
    s = np.sin(np.pi * k * (np.arange(N) + 1) * h)
    lam = float(np.sum(oracle.bspline(n, np.arange(-3, 4)) * np.cos(np.pi * k * np.arange(-3, 4) * h)))
    assert np.max(np.abs(B @ s - lam * s)) <= 1e-13
    assert np.max(np.abs(Bbad @ s - lam * s)) > 1e-3
