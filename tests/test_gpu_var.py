"""Variable-coefficient operator (Eq. tensForm with D and mu_a in B-splines) on the GPU vs the
FP64 oracle's plain triple sum, through the C ABI.

Operator tolerances (max norm, relative to max_i (|A(d, m)| |x|)_i): 1e-12 in FP64 and 1e-5 in
FP32, the FP32 case against the oracle applied to the FP32-rounded x, d and m that the kernel
reads. Grids span several output tiles with ragged tails in x and y and several z-blocks
(tiles: FP32 16 x 16 for degree <= 3, 12 x 12 and 10 x 10 for degrees 4 and 5; FP64 16, 12, 8,
8, 4 for degrees 1..5; z-blocks of at least 2n planes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1904_03057_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api as a
    return a


DIMS = {1: (37, 21, 19), 2: (35, 27, 13), 3: (37, 21, 19), 4: (19, 17, 11), 5: (13, 11, 10)}


def case(n, dims, seed, masked, aniso=True):
    nx, ny, nz = dims
    hs = (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1)) if aniso else (1 / (max(dims) + 1),) * 3
    mask = None
    if masked:
        mask = inputs.sphere_mask(nx, ny, nz, radius=0.42, h=hs).numpy()
        mask |= (np.random.default_rng(seed).random(mask.shape) < 0.05).astype(np.uint8)
    P = oracle.Problem(nx, ny, nz, n, *hs, dt=0.004, mask=mask)
    d = inputs.inclusion_coefficients(nx, ny, nz, seed=seed, h=hs).numpy()
    m = 1.0 + 0.5 * inputs.inclusion_coefficients(nx, ny, nz, seed=seed + 100, h=hs, base=0.3).numpy()
    x = inputs.random_field(P.shape, seed + 1).numpy()
    return P, hs, d, m, x


def make_handle(api, P, hs, precision):
    mask = None if P.mask is None else torch.from_numpy(P.mask).cuda()
    return api.Handle(P.nx, P.ny, P.nz, P.n, hs, P.dt, mask=mask, precision=precision)


def set_fields(H, d, m):
    H.set_coefficients(torch.from_numpy(d).cuda(), torch.from_numpy(m).cuda())


def f32r(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_op_apply_matches_oracle(api, prec, n):
    P, hs, d, m, x = case(n, DIMS[n], 10 + n, masked=(n % 2 == 1))
    H = make_handle(api, P, hs, prec)
    set_fields(H, d, m)
    dtype = torch.float64 if prec == "f64" else torch.float32
    y = H.op_apply(torch.from_numpy(x).to("cuda", dtype)).double().cpu().numpy()
    if prec == "f32":
        d, m, x = f32r(d), f32r(m), f32r(x)
    ref = oracle.op_var(P, d, m, x)
    scale = np.max(oracle.abs_op_var(P, d, m, x))
    tol = 1e-12 if prec == "f64" else 1e-5
    err = np.max(np.abs(y - ref)) / scale
    assert err <= tol, err
    if P.mask is not None:
        assert np.all(y[P.mask == 0] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unit_coefficients_match_constant_kernel(api, prec):
    """d = m = 1 gives the constant-coefficient operator: the variable-coefficient kernel agrees
    with the separable-sweep kernel of the same handle."""
    n, dims = 3, (48, 40, 36)
    P, hs, _, _, x = case(n, dims, 5, masked=True)
    H = make_handle(api, P, hs, prec)
    dtype = torch.float64 if prec == "f64" else torch.float32
    xt = torch.from_numpy(x).to("cuda", dtype)
    y0 = H.op_apply(xt).double().cpu().numpy()
    one = torch.ones(H.coef_shape, dtype=torch.float64, device="cuda")
    H.set_coefficients(one, one)
    y1 = H.op_apply(xt).double().cpu().numpy()
    H.set_coefficients(None, None)
    y2 = H.op_apply(xt).double().cpu().numpy()
    scale = np.max(oracle.abs_op(P, f32r(x) if prec == "f32" else x))
    tol = 1e-12 if prec == "f64" else 2e-5
    assert np.max(np.abs(y1 - y0)) <= tol * scale
    assert np.array_equal(y2, y0)


@pytest.mark.parametrize("n", [2, 3])
def test_minimum_axis_and_empty_mask(api, n):
    """Axes of n unknowns (the smallest the handle accepts: every ghost within one reflection)
    and a mask with no active node."""
    P, hs, d, m, x = case(n, (n, n + 1, n + 2), 40 + n, masked=False)
    H = make_handle(api, P, hs, "f64")
    set_fields(H, d, m)
    y = H.op_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.op_var(P, d, m, x)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(oracle.abs_op_var(P, d, m, x))
    P2, hs2, d2, m2, x2 = case(n, (20, 18, 9), 50 + n, masked=False)
    zero = torch.zeros((9, 18, 20), dtype=torch.uint8, device="cuda")
    H2 = api.Handle(20, 18, 9, n, hs2, P2.dt, mask=zero, precision="f32")
    set_fields(H2, d2, m2)
    y2 = H2.op_apply(torch.from_numpy(x2).cuda().float())
    assert torch.count_nonzero(y2).item() == 0


def test_sampled_parity_at_scale(api):
    """FP32, cubic, 256^3 with a masked domain and the inclusion fields: 300 sampled outputs
    against the oracle's definition at those points."""
    n, N = 3, 256
    h = 1.0 / (N + 1)
    mask_t = inputs.sphere_mask(N, N, N, radius=0.45, h=h, device="cuda")
    mask = mask_t.cpu().numpy()
    P = oracle.Problem(N, N, N, n, h, dt=5e-4, mask=mask)
    d = inputs.inclusion_coefficients(N, N, N, seed=7, h=h)
    m = 1.0 + 0.5 * inputs.inclusion_coefficients(N, N, N, seed=8, h=h, base=0.3)
    x = inputs.random_field((N, N, N), 9, device="cuda", dtype=torch.float32)
    H = api.Handle(N, N, N, n, h, 5e-4, mask=mask_t, precision="f32")
    H.set_coefficients(d.cuda(), m.cuda())
    y = H.op_apply(x).double().cpu().numpy().reshape(-1)
    rng = np.random.default_rng(3)
    act = np.flatnonzero(mask.reshape(-1))
    pts = np.concatenate([rng.choice(act, 280, replace=False), rng.choice(x.numel(), 20, replace=False)])
    xf = x.cpu().numpy()
    d32, m32 = f32r(d.numpy()), f32r(m.numpy())
    ref = oracle.op_var_points(P, d32, m32, xf, pts)
    scale = np.max(oracle.op_var_points(P, d32, m32, xf, pts, absolute=True))
    assert np.max(np.abs(y[pts] - ref)) <= 1e-5 * scale


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32_ir", 1e-8)])
def test_cg_solve_with_coefficients(api, prec, tol):
    """CG on A(d, m) x = b reaches the tolerance in the oracle's own FP64 residual."""
    n, dims = 3, (30, 26, 22)
    P, hs, d, m, _ = case(n, dims, 60, masked=True)
    b = inputs.random_field(P.shape, 61, mask=torch.from_numpy(P.mask)).numpy()
    H = make_handle(api, P, hs, prec)
    set_fields(H, d, m)
    x = torch.zeros(P.shape, dtype=torch.float64, device="cuda")
    rep = H.cg_solve(torch.from_numpy(b).cuda(), x, tol=tol, max_iter=5000)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol, rep
    xs = x.cpu().numpy()
    r = b * P.mask - oracle.op_var(P, d, m, xs)
    rel = np.linalg.norm(r) / np.linalg.norm(b * P.mask)
    assert rel <= 1.5 * tol, (rel, rep)


def test_heat_step_unit_coefficients_match_constant(api):
    """With d = m = 1, heat_step on the variable-coefficient operator gives the constant
    operator's implicit Euler steps."""
    n, dims = 3, (28, 24, 20)
    P, hs, _, _, _ = case(n, dims, 70, masked=True)
    u0 = inputs.random_field(P.shape, 71, mask=torch.from_numpy(P.mask)).cuda()
    out = []
    for var in (False, True):
        H = make_handle(api, P, hs, "f64")
        if var:
            one = torch.ones(H.coef_shape, dtype=torch.float64, device="cuda")
            H.set_coefficients(one, one)
        u = u0.clone()
        rep = H.heat_step(u, nsteps=3, tol=1e-11)
        assert rep["status"] == 0
        out.append(u)
    diff = (torch.linalg.vector_norm(out[1] - out[0]) / torch.linalg.vector_norm(out[0])).item()
    assert diff <= 1e-9


def test_fcg_without_network_on_coefficients(api):
    n, dims = 3, (24, 24, 24)
    P, hs, d, m, _ = case(n, dims, 80, masked=True)
    b = inputs.random_field(P.shape, 81, mask=torch.from_numpy(P.mask)).numpy()
    H = make_handle(api, P, hs, "f32_ir")
    set_fields(H, d, m)
    x = torch.zeros(P.shape, dtype=torch.float64, device="cuda")
    rep = H.fcg_solve(torch.from_numpy(b).cuda(), x, None, tol=1e-8)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-8
    r = b * P.mask - oracle.op_var(P, d, m, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b * P.mask) <= 1.5e-8


def test_argument_errors_and_flops(api):
    H = api.Handle(16, 16, 16, 3, 1 / 17, 1e-3, precision="f32")
    with pytest.raises(ValueError):
        H.set_coefficients(torch.ones((16, 16, 16), dtype=torch.float64, device="cuda"), None)
    a0, e0 = H.op_flops()
    assert a0 == e0 == 14 * 7
    H.set_coefficients(torch.ones(H.coef_shape, dtype=torch.float64, device="cuda"), None)
    a1, e1 = H.op_flops()
    assert 1e4 < a1 < e1
    B = api.Handle(16, 16, 16, 3, 1 / 17, 1e-3, precision="bf16s")
    with pytest.raises(Exception):
        B.set_coefficients(None, torch.ones(B.coef_shape, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32_ir", 1e-8)])
def test_jacobi_pcg_with_coefficients(api, prec, tol):
    """Jacobi PCG on A(d, m): the diagonal comes from probing the operator; the iteration matches
    the oracle's Jacobi PCG (whose diagonal is the triple-sum definition) and reaches the
    tolerance in the oracle's FP64 residual."""
    n, dims = 3, (30, 26, 22)
    P, hs, d, m, _ = case(n, dims, 90, masked=True)
    b = inputs.random_field(P.shape, 91, mask=torch.from_numpy(P.mask)).numpy()
    H = make_handle(api, P, hs, prec)
    set_fields(H, d, m)
    H.set_preconditioner("jacobi")
    x = torch.zeros(P.shape, dtype=torch.float64, device="cuda")
    rep = H.cg_solve(torch.from_numpy(b).cuda(), x, tol=tol, max_iter=5000)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol, rep
    r = b * P.mask - oracle.op_var(P, d, m, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b * P.mask) <= 1.5 * tol
    if prec == "f64":
        _, it_ref, _, st = oracle.pcg_var(P, d, m, b, tol=tol)
        assert st == 0 and abs(rep["iterations"] - it_ref) <= 3, (rep["iterations"], it_ref)
        # plain CG on the same system takes more iterations (the fields vary by a factor 25)
        x2 = torch.zeros_like(x)
        H.set_preconditioner("none")
        rep2 = H.cg_solve(torch.from_numpy(b).cuda(), x2, tol=tol, max_iter=5000)
        assert rep2["status"] == 0 and rep["iterations"] < rep2["iterations"], (rep, rep2)


def test_heat_step_with_coefficients(api):
    """One implicit Euler step A(d, m) u1 = M u0 (constant mass on the right-hand side) against
    the oracle's Jacobi PCG on the variable-coefficient system."""
    n, dims = 3, (26, 22, 18)
    P, hs, d, m, _ = case(n, dims, 95, masked=True)
    u0 = inputs.random_field(P.shape, 96, mask=torch.from_numpy(P.mask)).numpy()
    b = oracle.mass(P, u0)
    ref, _, _, st = oracle.pcg_var(P, d, m, b, tol=1e-12)
    assert st == 0
    H = make_handle(api, P, hs, "f64")
    set_fields(H, d, m)
    u = torch.from_numpy(u0).cuda()
    rep = H.heat_step(u, nsteps=1, tol=1e-11)
    assert rep["status"] == 0
    got = u.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
