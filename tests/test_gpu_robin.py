"""Boundary-penalty (Robin) problems, Jacobi-preconditioned CG and the coarse-to-fine
prolongation on the GPU against the FP64 oracle, through the C ABI.

Operator tolerances as for the other operators (1e-12 FP64, 1e-5 FP32 of the |A||x| scale).
Robin grids: the handle's dimensions are the unknowns of the untruncated basis,
N + 2 + 2 floor(n/2) for a box of N interior nodes; the general kernel's 32 x 16 tiles and
z-blocks of at least 16 planes are spanned with ragged tails."""
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


INTERIOR = {1: (37, 19, 34), 2: (35, 21, 33), 3: (37, 19, 31), 4: (29, 17, 27), 5: (27, 15, 25)}


def robin_case(api, n, N, prec, pen, dt=0.02, seed=0):
    hs = tuple(1.0 / (k + 1) for k in N)
    P = oracle.Problem(*N, n, *hs, dt=dt)
    shape = oracle.robin_shape(P)
    H = api.Handle(shape[2], shape[1], shape[0], n, hs, dt, precision=prec)
    H.set_boundary("robin", pen)
    x = np.random.default_rng(seed).standard_normal(shape)
    return P, H, x


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_robin_operator_matches_oracle(api, prec, n):
    P, H, x = robin_case(api, n, INTERIOR[n], prec, pen=7.5, seed=n)
    dt = torch.float64 if prec == "f64" else torch.float32
    xx = x if prec == "f64" else x.astype(np.float32).astype(np.float64)
    y = H.op_apply(torch.from_numpy(x).to("cuda", dt)).double().cpu().numpy()
    ref = oracle.op_robin(P, 7.5, xx)
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.max(np.abs(y - ref)) <= tol * np.max(oracle.abs_op_robin(P, 7.5, xx))
    m = H.mass_apply(torch.from_numpy(x).to("cuda", dt)).double().cpu().numpy()
    P0 = oracle.Problem(*INTERIOR[n], n, P.hx, P.hy, P.hz, dt=0.0)
    refm = oracle.op_robin(P0, 0.0, xx)
    assert np.max(np.abs(m - refm)) <= tol * np.max(oracle.abs_op_robin(P0, 0.0, xx))


@pytest.mark.parametrize("n,pc", [(1, "none"), (1, "jacobi"), (3, "jacobi")])
def test_robin_cg_solve(api, n, pc):
    """CG / Jacobi PCG on A_R x = b reaches the tolerance in the oracle's own FP64 residual."""
    N = (20, 17, 22)
    P, H, _ = robin_case(api, n, N, "f64", pen=50.0, dt=0.01)
    H.set_preconditioner(pc)
    b = inputs.random_field(oracle.robin_shape(P), 3).numpy()
    x = torch.zeros(oracle.robin_shape(P), dtype=torch.float64, device="cuda")
    rep = H.cg_solve(torch.from_numpy(b).cuda(), x, tol=1e-9, max_iter=20000)
    assert rep["status"] == 0, rep
    r = b - oracle.op_robin(P, 50.0, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 3e-9
    if pc == "jacobi":
        # same preconditioned iteration in the oracle; rounding shifts the count a little on
        # this ill-conditioned basis
        _, it_ref, _, st = oracle.pcg(P, b, tol=1e-9, pen=50.0, robin=True, max_iter=20000)
        assert st == 0 and abs(rep["iterations"] - it_ref) <= 0.25 * it_ref + 5, (rep["iterations"], it_ref)


@pytest.mark.parametrize("prec", ["f64", "f32_ir"])
def test_jacobi_pcg_dirichlet_masked(api, prec):
    """Jacobi PCG on the masked Dirichlet operator: same iteration count as the oracle's PCG,
    solution within the FP64 residual the oracle measures."""
    n, N = 3, (30, 26, 22)
    hs = tuple(1.0 / (k + 1) for k in N)
    mask = inputs.sphere_mask(*N, radius=0.42, h=hs).numpy()
    P = oracle.Problem(*N, n, *hs, dt=0.004, mask=mask)
    b = inputs.random_field(P.shape, 5, mask=torch.from_numpy(mask)).numpy()
    H = api.Handle(*N, n, hs, 0.004, mask=torch.from_numpy(mask).cuda(), precision=prec)
    H.set_preconditioner("jacobi")
    x = torch.zeros(P.shape, dtype=torch.float64, device="cuda")
    tol = 1e-10 if prec == "f64" else 1e-8
    rep = H.cg_solve(torch.from_numpy(b).cuda(), x, tol=tol)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol
    r = b - oracle.op_stencil(P, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5 * tol
    if prec == "f64":
        _, it_ref, _, st = oracle.pcg(P, b, tol=tol)
        assert st == 0 and abs(rep["iterations"] - it_ref) <= 3, (rep["iterations"], it_ref)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_prolongation_matches_oracle(api, n):
    Nc, Nf = (9, 7, 11), (19, 15, 23)      # coarse step 2 h: nested grids
    hc = tuple(1.0 / (k + 1) for k in Nc)
    hf = tuple(1.0 / (k + 1) for k in Nf)
    C = oracle.Problem(*Nc, n, *hc, dt=0.0)
    F = oracle.Problem(*Nf, n, *hf, dt=0.0)
    sc, sf = oracle.robin_shape(C), oracle.robin_shape(F)
    Hc = api.Handle(sc[2], sc[1], sc[0], n, hc, 0.0, precision="f64")
    Hf = api.Handle(sf[2], sf[1], sf[0], n, hf, 0.0, precision="f64")
    Hc.set_boundary("robin", 1.0)
    Hf.set_boundary("robin", 1.0)
    xc = np.random.default_rng(n).standard_normal(sc)
    xf = api.prolong(Hf, Hc, torch.from_numpy(xc).cuda()).cpu().numpy()
    ref = oracle.prolong_robin(F, C, xc)
    assert np.max(np.abs(xf - ref)) <= 1e-9 * np.max(np.abs(ref))
    # a box mismatch is refused
    Hbad = api.Handle(sc[2] + 1, sc[1], sc[0], n, hc, 0.0, precision="f64")
    Hbad.set_boundary("robin", 1.0)
    with pytest.raises(Exception):
        api.prolong(Hf, Hbad, torch.zeros(Hbad.shape, dtype=torch.float64, device="cuda"))


def test_coarse_start_saves_iterations(api):
    """The coarse-grid start: a Robin problem solved on a grid of twice the step and prolonged
    is already close to the fine solution, and after a fixed number of fine Jacobi-PCG
    iterations (the paper ran its large problem for a fixed count) it stays well ahead of the
    start from zero; both reach the same answer. Errors are measured against the converged
    fine solution (the residual norm is dominated by the high frequencies that a coarse grid
    cannot represent)."""
    n, pen, dt = 1, 20.0, 0.02
    Nc, Nf = (15, 15, 31), (31, 31, 63)
    hc = tuple(1.0 / (k + 1) for k in Nc)
    hf = tuple(1.0 / (k + 1) for k in Nf)
    sc = tuple(api.robin_size(n, k) for k in reversed(Nc))
    sf = tuple(api.robin_size(n, k) for k in reversed(Nf))
    Hc = api.Handle(sc[2], sc[1], sc[0], n, hc, dt, precision="f64")
    Hf = api.Handle(sf[2], sf[1], sf[0], n, hf, dt, precision="f64")
    for H in (Hc, Hf):
        H.set_boundary("robin", pen)
        H.set_preconditioner("jacobi")
    # the same smooth source on both grids: a Gaussian sampled at the B-spline centres
    # ((a - floor(n/2)) h for unknown a; the generator samples at (a + 1) h, hence the shifted
    # centre), loaded with each grid's mass matrix
    def load(H, N, h, shape):
        off = [(1 + n // 2) * hh for hh in h]
        cs = [(0.5 + off[0], 0.45 + off[1], 0.6 + off[2])]
        q = inputs.gaussian_source(*[s for s in reversed(shape)], cs, sigma=0.15,
                                   h=h, device="cuda")
        return H.mass_apply(q)
    bc = load(Hc, Nc, hc, sc)
    bf = load(Hf, Nf, hf, sf)
    xc = torch.zeros(sc, dtype=torch.float64, device="cuda")
    assert Hc.cg_solve(bc, xc, tol=1e-8)["status"] == 0
    x0 = api.prolong(Hf, Hc, xc)
    xs = torch.zeros_like(x0)
    assert Hf.cg_solve(bf, xs, tol=1e-11)["status"] == 0
    err = lambda v: (torch.linalg.vector_norm(v - xs) / torch.linalg.vector_norm(xs)).item()
    assert err(x0) <= 0.1, err(x0)
    fixed = {}
    for name, start in (("warm", x0), ("cold", torch.zeros_like(x0))):
        x = start.clone()
        Hf.cg_solve(bf, x, tol=1e-14, max_iter=40)
        fixed[name] = err(x)
    assert fixed["warm"] < 0.2 * fixed["cold"], fixed
    x1 = x0.clone()
    r_warm = Hf.cg_solve(bf, x1, tol=1e-9)
    x2 = torch.zeros_like(x0)
    r_cold = Hf.cg_solve(bf, x2, tol=1e-9)
    assert r_warm["status"] == 0 and r_cold["status"] == 0
    assert r_warm["iterations"] <= r_cold["iterations"], (r_warm, r_cold)
    assert (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x2)).item() <= 1e-6


def test_argument_errors(api):
    H = api.Handle(20, 20, 20, 3, 1 / 17, 1e-3, mask=torch.ones((20, 20, 20), dtype=torch.uint8, device="cuda"))
    with pytest.raises(Exception):
        H.set_boundary("robin", 1.0)              # masks take the Dirichlet boundary
    H2 = api.Handle(20, 20, 20, 3, 1 / 17, 1e-3)
    H2.set_coefficients(torch.ones(H2.coef_shape, dtype=torch.float64, device="cuda"), None)
    with pytest.raises(Exception):
        H2.set_boundary("robin", 1.0)
    H2.set_preconditioner("jacobi")            # variable coefficients: probed diagonal
    H3 = api.Handle(20, 20, 20, 3, 1 / 17, 1e-3)
    x = inputs.random_field((20, 20, 20), 13).cuda()
    y_dir = H3.op_apply(x).clone()
    H3.set_boundary("robin", 1.0)
    with pytest.raises(Exception):
        H3.to_samples(torch.zeros((20, 20, 20), dtype=torch.float64, device="cuda"))
    with pytest.raises(Exception):
        H3.set_boundary("robin", -1.0)
    assert not torch.equal(H3.op_apply(x), y_dir)
    H3.set_boundary("dirichlet")              # back to the reflected basis: same operator again
    assert torch.equal(H3.op_apply(x), y_dir)
    H3.to_samples(torch.zeros((20, 20, 20), dtype=torch.float64, device="cuda"))


def test_robin_heat_step_and_mixed_precision(api):
    """One implicit Euler step on a Robin handle, (M + dt K + pen E) u1 = M u0 with the
    truncated mass M, against the oracle's Jacobi PCG on the same system; and the same system
    solved by FP32 inner PCG inside FP64 refinement."""
    n, N, pen, dt = 1, (22, 19, 25), 30.0, 0.01
    hs = tuple(1.0 / (k + 1) for k in N)
    P = oracle.Problem(*N, n, *hs, dt=dt)
    P0 = oracle.Problem(*N, n, *hs, dt=0.0)
    shape = oracle.robin_shape(P)
    u0 = inputs.random_field(shape, 12).numpy()
    b = oracle.op_robin(P0, 0.0, u0)                          # M u0
    ref, _, rel, st = oracle.pcg(P, b, tol=1e-12, pen=pen, robin=True, max_iter=20000)
    assert st == 0
    for prec, tol in (("f64", 1e-10), ("f32_ir", 1e-9)):
        H = api.Handle(shape[2], shape[1], shape[0], n, hs, dt, precision=prec)
        H.set_boundary("robin", pen)
        H.set_preconditioner("jacobi")
        u = torch.from_numpy(u0).cuda()
        rep = H.heat_step(u, nsteps=1, tol=tol, max_iter=20000)
        assert rep["status"] == 0, rep
        got = u.cpu().numpy()
        # the oracle's own true residual of the returned step, against the requested tolerance
        res = b - oracle.op_robin(P, pen, got)
        assert np.linalg.norm(res) <= 1.5 * tol * np.linalg.norm(b), (prec, rep)
        # and the error, bounded by the condition number times that residual (moderate here)
        assert np.linalg.norm(got - ref) <= 1e4 * tol * np.linalg.norm(ref), (prec, rep)


def test_prolongation_fp32(api):
    n = 3
    Nc, Nf = (9, 7, 11), (19, 15, 23)
    hc = tuple(1.0 / (k + 1) for k in Nc)
    hf = tuple(1.0 / (k + 1) for k in Nf)
    C = oracle.Problem(*Nc, n, *hc, dt=0.0)
    F = oracle.Problem(*Nf, n, *hf, dt=0.0)
    sc, sf = oracle.robin_shape(C), oracle.robin_shape(F)
    Hc = api.Handle(sc[2], sc[1], sc[0], n, hc, 0.0, precision="f32")
    Hf = api.Handle(sf[2], sf[1], sf[0], n, hf, 0.0, precision="f32")
    Hc.set_boundary("robin", 1.0)
    Hf.set_boundary("robin", 1.0)
    xc = np.random.default_rng(4).standard_normal(sc).astype(np.float32)
    xf = api.prolong(Hf, Hc, torch.from_numpy(xc).cuda()).double().cpu().numpy()
    ref = oracle.prolong_robin(F, C, xc.astype(np.float64))
    # computed in FP64 inside and rounded once to FP32
    assert np.max(np.abs(xf - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_robin_sampled_parity_at_scale(api):
    """FP64 linear Robin operator on 200 x 200 x 800 unknowns (0.2 G-node box of the large-run
    analogue's shape at a third of its size): 300 sampled outputs, the faces and corners
    included, against the oracle's band sum at those points."""
    n, pen, dt = 1, 1.0e3, 1.0
    nt = (200, 200, 800)
    N = tuple(k - 2 for k in nt)
    h = 1.0 / (nt[2] - 1)
    P = oracle.Problem(*N, n, h, dt=dt)
    H = api.Handle(*nt, n, h, dt, precision="f64")
    H.set_boundary("robin", pen)
    x = inputs.random_field((nt[2], nt[1], nt[0]), 14, device="cuda")
    y = H.op_apply(x).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(15)
    corners = [((z * nt[1] + yy) * nt[0] + xx) for z in (0, nt[2] - 1) for yy in (0, nt[1] - 1) for xx in (0, nt[0] - 1)]
    faces = [((rng.integers(nt[2]) * nt[1] + rng.integers(nt[1])) * nt[0] + f) for f in (0, 1, nt[0] - 2, nt[0] - 1)
             for _ in range(8)]
    pts = np.unique(np.concatenate([rng.choice(x.numel(), 260, replace=False), corners, faces]))
    xh = x.cpu().numpy()
    ref = oracle.op_robin_points(P, pen, xh, pts)
    scale = np.max(oracle.op_robin_points(P, pen, xh, pts, absolute=True))
    assert np.max(np.abs(y[pts] - ref)) <= 1e-12 * scale


@pytest.mark.parametrize("case", ["dirichlet", "dirichlet-masked", "robin"])
def test_inverse_diagonal_matches_oracle(api, case):
    """bsk_inverse_diagonal: 1 / diag A per node against the oracle's diagonal (FP64, 1e-13),
    including the nodes whose mirror images touch the faces, masked nodes (0) and the Robin
    boundary rows."""
    n, N = 3, (23, 17, 14)
    hs = tuple(1.0 / (k + 1) for k in N)
    mask = None
    if case == "robin":
        P = oracle.Problem(*N, n, *hs, dt=0.02)
        shape = oracle.robin_shape(P)
        H = api.Handle(shape[2], shape[1], shape[0], n, hs, 0.02, precision="f64")
        H.set_boundary("robin", 50.0)
        d = oracle.diag(P, pen=50.0, robin=True)
    else:
        if case == "dirichlet-masked":
            mask = (np.random.default_rng(3).random((N[2], N[1], N[0])) < 0.7).astype(np.uint8)
        P = oracle.Problem(*N, n, *hs, dt=0.02, mask=mask)
        H = api.Handle(*N, n, hs, 0.02, precision="f64",
                       mask=None if mask is None else torch.from_numpy(mask).cuda())
        d = oracle.diag(P)
    H.set_preconditioner("jacobi")
    inv = H.inverse_diagonal().cpu().numpy()
    want = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
    if mask is not None:
        assert np.all(inv[mask == 0] == 0.0)
        act = mask != 0
        assert np.allclose(inv[act], want[act], rtol=1e-13, atol=0)
    else:
        assert np.allclose(inv, want, rtol=1e-13, atol=0)
    H.close()
