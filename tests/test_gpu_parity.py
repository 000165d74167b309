"""CUDA path vs the FP64 oracle, through the C ABI (Python binding -> libbsk.so).

Operator tolerances (max norm, relative to max_i (|A| |x|)_i, the size of the terms summed):
1e-12 in FP64 and 1e-5 in FP32. Solves are judged by the oracle's FP64 true residual of the
GPU solution and by the distance to the oracle solution, bounded by kappa * tol with kappa the
condition number of the box operator (an upper bound for masked domains, whose matrices are
principal submatrices)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1904_03057_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

from test_oracle_pins import exact_kernels, symbol  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api as a
    return a


def box_kappa(nx, ny, nz, n, hs, dt):
    """Condition number of the box operator from its sine-mode eigenvalues."""
    me, ke = exact_kernels(n)
    lam_m, lam_k = [], []
    for N, h in zip((nx, ny, nz), hs):
        th = np.pi * np.arange(1, N + 1) * h
        js = np.arange(-n, n + 1)
        mh = h * np.array([float(v) for v in me]) @ np.cos(np.outer(js, th))
        kh = np.array([float(v) for v in ke]) @ np.cos(np.outer(js, th)) / h
        lam_m.append(mh)
        lam_k.append(kh)
    mx, my = np.meshgrid(lam_m[0], lam_m[1], indexing="ij")
    kx, ky = np.meshgrid(lam_k[0], lam_k[1], indexing="ij")
    lo, hi = np.inf, 0.0
    for mz, kz in zip(lam_m[2], lam_k[2]):   # one z mode at a time (bounded memory)
        lam = mx * my * mz + dt * (kx * my * mz + mx * ky * mz + mx * my * kz)
        lo, hi = min(lo, lam.min()), max(hi, lam.max())
    return float(hi / lo)


def make_problem(orc, nx, ny, nz, n, dt, masked, seed=0, hs=None):
    hs = hs or (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1))
    mask = None
    if masked:
        mask = inputs.sphere_mask(nx, ny, nz, radius=0.42, h=hs).numpy()
        mask |= (np.random.default_rng(seed).random(mask.shape) < 0.05).astype(np.uint8)
    return orc.Problem(nx, ny, nz, n, *hs, dt=dt, mask=mask), hs


def handle(api, p, hs, precision):
    m = None if p.mask is None else torch.from_numpy(p.mask).cuda()
    return api.Handle(p.nx, p.ny, p.nz, p.n, hs, p.dt, mask=m, precision=precision)


OP_CASES = [
    # nx, ny, nz, n, dt, masked -- several 32 x 16 tiles with ragged tails, several z chunks
    (70, 37, 41, 3, 1e-3, False),
    (33, 33, 33, 1, 0.05, True),
    (45, 20, 18, 2, 0.01, True),
    (40, 17, 35, 4, 2e-3, False),
    (36, 36, 20, 5, 5e-4, True),
    (1, 1, 1, 1, 0.3, False),
    (2, 3, 2, 2, 0.1, False),
    (3, 3, 4, 3, 0.1, True),
    (4, 5, 4, 4, 0.1, False),
    (5, 5, 6, 5, 0.1, False),
    # unmasked grids with 16-byte rows take the TMA kernels: 64 x 32 tiles for the FP32 operator
    # (64 x 24 for the other passes), ragged x / y / z
    (68, 5120, 8, 3, 1e-3, False),   # 160 tiles: blocks take two items; loads run across items
    (196, 70, 45, 3, 2e-3, False),
    (64, 32, 300, 2, 5e-3, False),   # several z-chunks per tile
    (68, 50, 30, 1, 0.02, False),
    (68, 50, 30, 2, 0.01, False),
    (68, 50, 31, 3, 1e-3, False),
    (132, 49, 27, 4, 2e-3, False),
    (72, 26, 19, 5, 5e-4, False),
    (4, 4, 4, 3, 0.1, False),
    (8, 30, 5, 5, 0.1, False),
    (64, 24, 9, 3, 0.1, False),
]


@pytest.mark.parametrize("nx,ny,nz,n,dt,masked", OP_CASES)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_op_apply_matches_oracle(api, orc, nx, ny, nz, n, dt, masked, precision):
    p, hs = make_problem(orc, nx, ny, nz, n, dt, masked, seed=nx)
    x = np.random.default_rng(nx * 7 + n).standard_normal(p.shape)
    H = handle(api, p, hs, precision)
    tdt = torch.float64 if precision == "f64" else torch.float32
    xt = torch.from_numpy(x).to("cuda", tdt)
    xin = xt.double().cpu().numpy()          # the exact input values the GPU saw
    y = H.op_apply(xt).double().cpu().numpy()
    ref = orc.op_separable(p, xin)
    scale = np.max(orc.abs_op(p, xin))
    tol = 1e-12 if precision == "f64" else 1e-5
    assert np.max(np.abs(y - ref)) <= tol * scale
    if p.mask is not None:
        assert np.all(y[p.mask == 0] == 0)
    # mass operator alone
    ym = H.mass_apply(xt).double().cpu().numpy()
    pm = orc.Problem(p.nx, p.ny, p.nz, p.n, *hs, dt=0.0, mask=p.mask)
    refm = orc.mass(pm, xin)
    assert np.max(np.abs(ym - refm)) <= tol * np.max(orc.abs_op(pm, xin))


def test_op_apply_does_not_read_masked_inputs(api, orc):
    p, hs = make_problem(orc, 30, 20, 25, 3, 1e-3, True)
    x = np.random.default_rng(3).standard_normal(p.shape)
    H = handle(api, p, hs, "f64")
    y1 = H.op_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    x2 = x.copy()
    x2[p.mask == 0] = 1e30
    y2 = H.op_apply(torch.from_numpy(x2).cuda()).cpu().numpy()
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-5), ("f32_ir", 1e-10)])
@pytest.mark.parametrize("masked,nx", [(False, 37), (True, 37), (False, 44)])
def test_cg_solve_matches_oracle(api, orc, precision, tol, masked, nx):
    """nx = 44 (16-byte rows, unmasked) runs the single-pass TMA iteration; nx = 37 and masked
    grids run the general kernels."""
    ny, nz, n, dt = 29, 23, 3, 2e-3
    p, hs = make_problem(orc, nx, ny, nz, n, dt, masked, seed=4)
    b = np.random.default_rng(11).standard_normal(p.shape)
    if p.mask is not None:
        b *= p.mask
    H = handle(api, p, hs, precision)
    tdt = torch.float32 if precision == "f32" else torch.float64
    bt = torch.from_numpy(b).to("cuda", tdt)
    xt = torch.zeros_like(bt)
    rep = H.cg_solve(bt, xt, tol=tol, max_iter=5000)
    assert rep["status"] == 0
    x = xt.double().cpu().numpy()
    bin_ = bt.double().cpu().numpy()
    r = bin_ - orc.op_separable(p, x)
    true_rel = np.linalg.norm(r) / np.linalg.norm(bin_)
    assert true_rel <= (10 * tol if precision == "f32" else 1.5 * tol)
    assert abs(rep["rel_residual"] - true_rel) <= 0.05 * true_rel + 1e-6 * (precision == "f32")
    xr, it, rel, st = orc.cg(p, bin_, tol=1e-13, max_iter=5000)
    kappa = box_kappa(nx, ny, nz, n, hs, dt)
    err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
    assert err <= kappa * true_rel * 1.01 + 1e-12
    if precision == "f64":
        _, it_o, _, _ = orc.cg(p, bin_, tol=tol, max_iter=5000)
        assert abs(rep["iterations"] - it_o) <= 3
    if p.mask is not None:
        assert np.all(x[p.mask == 0] == 0)


TMA_CG_CASES = [
    # nx, ny, nz, n, isotropic -- unmasked 16-byte rows: the single-pass iteration on 64 x 32 tiles
    (132, 70, 40, 3, True),     # ragged tiles in x and y
    (132, 70, 40, 3, False),    # anisotropic steps: four z tap sets
    (68, 2600, 6, 2, True),     # 164 tiles: blocks take two items
    (68, 40, 30, 4, False),
    (64, 32, 150, 1, True),     # several z-chunks per tile
]


@pytest.mark.parametrize("nx,ny,nz,n,iso", TMA_CG_CASES)
@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f32_ir", 1e-10)])
@pytest.mark.parametrize("kernel", ["ws_chunked", "ws_columns", "classic"])
def test_cg_solve_tma_tiles_matches_oracle(api, orc, nx, ny, nz, n, iso, precision, tol, kernel):
    """The single-pass CG iteration, with each of its two kernels (the warp-specialised one with
    chunked and with whole-column items), on grids spanning several tiles,
    items and z-chunks, judged by the oracle's FP64 true residual of the returned solution and its
    distance to the oracle's solution (kappa times the residual)."""
    dt = 2e-3
    h = 1 / (max(nx, ny, nz) + 1)
    hs = (h, h, h) if iso else (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1))
    p = orc.Problem(nx, ny, nz, n, *hs, dt=dt)
    b = np.random.default_rng(nx + ny + n).standard_normal(p.shape)
    H = handle(api, p, hs, precision)
    assert H.select_cg_kernel(kernel) == ("classic" if kernel == "classic" else "ws")
    tdt = torch.float32 if precision == "f32" else torch.float64
    bt = torch.from_numpy(b).to("cuda", tdt)
    xt = torch.zeros_like(bt)
    rep = H.cg_solve(bt, xt, tol=tol, max_iter=5000)
    assert rep["status"] == 0, rep
    x = xt.double().cpu().numpy()
    bin_ = bt.double().cpu().numpy()
    r = bin_ - orc.op_separable(p, x)
    true_rel = np.linalg.norm(r) / np.linalg.norm(bin_)
    assert true_rel <= (10 * tol if precision == "f32" else 1.5 * tol), true_rel
    xr, _, _, _ = orc.cg(p, bin_, tol=1e-13, max_iter=5000)
    kappa = box_kappa(nx, ny, nz, n, hs, dt)
    err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
    assert err <= kappa * true_rel * 1.01 + 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32", "f32_ir"])
@pytest.mark.parametrize("nx", [37, 68])
def test_cg_stall_status(api, precision, nx):
    """The plain-CG stall test (no new smallest residual within stall_window iterations). On the
    mass matrix alone (dt = 0: an L2 projection) the 2-norm of the CG residual rises at the first
    iteration (checked with the oracle's operator in a plain CG), so a window of one or two trips
    it: the solve must end with status 2 (stalled) or 0 (converged first) after a bounded number
    of iterations, never hang. Under FP64 refinement a stalled inner solve only ends that inner
    solve; the refinement goes on and ends converged (0) or out of refinement steps (1)."""
    n, dt = 3, 0.0
    h = 1 / (nx + 1)
    H = api.Handle(nx, 30, 26, n, h, dt, precision=precision)
    tdt = torch.float32 if precision == "f32" else torch.float64
    b = torch.from_numpy(np.random.default_rng(5).standard_normal((26, 30, nx))).to("cuda", tdt)
    x = torch.zeros_like(b)
    allowed = (0, 1) if precision == "f32_ir" else (0, 2)
    statuses = set()
    for window in (1, 2):
        rep = H.cg_solve(b, torch.zeros_like(b), tol=1e-12, max_iter=4000, stall_window=window)
        assert rep["status"] in allowed, rep
        assert rep["iterations"] <= 4000 and math.isfinite(rep["rel_residual"])
        statuses.add(rep["status"])
    if precision != "f32_ir":
        assert 2 in statuses, "a window of one or two iterations should trip on a CG residual"


def test_cg_kernel_selection(api):
    """bsk_select_cg_kernel: AUTO picks one of the two kernels; the warp-specialised pass is
    refused where it does not apply (masked grid, FP64, degree 5); a forced choice sticks."""
    H = api.Handle(68, 40, 20, 3, 1 / 69, 1e-3, precision="f32_ir")
    assert H.select_cg_kernel("auto") in ("ws", "classic")
    assert H.select_cg_kernel("classic") == "classic"
    assert H.select_cg_kernel("ws") == "ws"
    assert H.select_cg_kernel("current") == "ws"
    assert H.cg_kernel_config()["zchunk_planes"] in (128, 20)
    assert H.select_cg_kernel("ws_columns") == "ws" and H.cg_kernel_config() == {"kernel": "ws", "zchunk_planes": 20}
    assert H.select_cg_kernel("ws_chunked") == "ws" and H.cg_kernel_config() == {"kernel": "ws", "zchunk_planes": 128}
    assert H.select_cg_kernel("classic") == "classic" and H.cg_kernel_config()["zchunk_planes"] == 0
    for kw in (dict(precision="f64"), dict(precision="f32", degree=5),
               dict(precision="f32", mask=torch.ones((20, 40, 68), dtype=torch.uint8, device="cuda"))):
        deg = kw.pop("degree", 3)
        Hx = api.Handle(68, 40, 20, deg, 1 / 69, 1e-3, **kw)
        for req in ("ws", "ws_chunked", "ws_columns"):
            with pytest.raises(RuntimeError, match="-1"):
                Hx.select_cg_kernel(req)
        assert Hx.select_cg_kernel("auto") == "classic"


def test_heat_step_32cube_closed_form(api, orc):
    """32^3, cubic, sin sin sin initial coefficients, dt = 1e-3, 10 steps, tol 1e-10, FP64."""
    N, n, dt, K, tol = 32, 3, 1e-3, 10, 1e-10
    h = 1 / (N + 1)
    u0 = inputs.sine_mode_field(N, N, N, [((1, 1, 1), 1.0)])
    H = api.Handle(N, N, N, n, h, dt, precision="f64")
    u = u0.cuda().clone()
    rep = H.heat_step(u, None, K, tol=tol)
    assert rep["status"] == 0
    me, ke = exact_kernels(n)
    mh, kh = h * symbol(me, math.pi * h), symbol(ke, math.pi * h) / h
    g = mh ** 3 / (mh ** 3 + 3 * dt * kh * mh ** 2)
    want = (g ** K) * u0.numpy()
    got = u.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(u0.numpy())) * K
    p = orc.Problem(N, N, N, n, h, dt=dt)
    ur, its, rel, st = orc.heat(p, u0.numpy(), None, K, tol=tol)
    assert np.max(np.abs(got - ur)) <= 1e-12
    assert rep["iterations"] == K  # one eigenvector: one CG iteration per step


def test_heat_step_masked_gaussian_sources_fp64_vs_ir(api, orc):
    """A reduced sphere-masked heat problem: sphere mask r = 0.45, 32 Gaussian sources (sigma 0.03, seed 2),
    u0 = 0, dt = 1e-3, a few steps; FP64 CG vs FP32-sweep + FP64 refinement vs the oracle."""
    N, n, dt, K, tol = 48, 3, 1e-3, 3, 1e-10
    h = 1 / (N + 1)
    mask = inputs.sphere_mask(N, N, N, radius=0.45)
    q = inputs.gaussian_source(N, N, N, inputs.gaussian_centers(2, 32), 0.03, mask=mask)
    res = {}
    for prec in ("f64", "f32_ir"):
        H = api.Handle(N, N, N, n, h, dt, mask=mask.cuda(), precision=prec)
        u = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
        rep = H.heat_step(u, q.cuda(), K, tol=tol)
        assert rep["status"] == 0
        res[prec] = u.cpu().numpy()
    p = orc.Problem(N, N, N, n, h, dt=dt, mask=mask.numpy())
    ur, its, rel, st = orc.heat(p, np.zeros(p.shape), q.numpy(), K, tol=1e-13)
    kappa = box_kappa(N, N, N, n, (h, h, h), dt)
    for prec, u in res.items():
        err = np.linalg.norm(u - ur) / np.linalg.norm(ur)
        assert err <= 2 * K * kappa * tol, (prec, err)
    d = np.linalg.norm(res["f64"] - res["f32_ir"]) / np.linalg.norm(res["f64"])
    assert d <= 4 * K * kappa * tol


def test_cg_edge_cases(api, orc):
    N, n = 20, 2
    h = 1 / (N + 1)
    H = api.Handle(N, N, N, n, h, 1e-3, precision="f64")
    b = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    x = torch.randn_like(b)
    rep = H.cg_solve(b, x)
    assert rep["status"] == 0 and rep["iterations"] == 0
    assert torch.count_nonzero(x).item() == 0  # b = 0 gives x = 0
    b = torch.randn_like(b)
    x = torch.zeros_like(b)
    rep = H.cg_solve(b, x, tol=1e-12, max_iter=1)
    assert rep["status"] == 1 and rep["iterations"] == 1
    # warm start from a converged solution: no iterations
    x = torch.zeros_like(b)
    H.cg_solve(b, x, tol=1e-9)
    rep = H.cg_solve(b, x, tol=1e-9)
    assert rep["status"] == 0 and rep["iterations"] == 0
    # NaN in the right-hand side: breakdown reported, no hang
    bn = b.clone()
    bn[3, 4, 5] = float("nan")
    with pytest.raises(RuntimeError, match="-5"):
        H.cg_solve(bn, torch.zeros_like(b))
    # wall-clock limit
    with pytest.raises(RuntimeError, match="-4"):
        H.cg_solve(b, torch.zeros_like(b), tol=1e-300, max_iter=10 ** 6, time_limit_s=1e-6,
                   check_every=2)
    # all-inactive mask
    Hm = api.Handle(N, N, N, n, h, 1e-3, mask=torch.zeros((N, N, N), dtype=torch.uint8,
                                                          device="cuda"), precision="f64")
    y = Hm.op_apply(b)
    assert torch.count_nonzero(y).item() == 0
    x = torch.ones_like(b)
    rep = Hm.cg_solve(b, x)
    assert rep["status"] == 0 and torch.count_nonzero(x).item() == 0
    # wrong dtype / shape are rejected by the binding, overlapping vectors by the library
    with pytest.raises(ValueError):
        H.op_apply(b.float())
    with pytest.raises(RuntimeError, match="-1"):
        H.op_apply(b, b)


def test_full_size_928_operator_sampled_and_eigen(api, orc):
    """928^3 FP32 op_apply (the benchmark's launch configuration): every output against the
    sine-mode eigen-relation, and 3000 sampled outputs (faces, edges, corners included) of a
    64-mode field against the oracle evaluated point by point."""
    N, n, dt = 928, 3, 5e-4
    h = 1 / (N + 1)
    H = api.Handle(N, N, N, n, h, dt, precision="f32")
    me, ke = exact_kernels(n)
    kv = (3, 1, 7)
    x = inputs.sine_mode_field(N, N, N, [(kv, 1.0)], device="cuda", dtype=torch.float32)
    y = H.op_apply(x)
    mh = [h * symbol(me, math.pi * k * h) for k in kv]
    kh = [symbol(ke, math.pi * k * h) / h for k in kv]
    lam = mh[0] * mh[1] * mh[2] + dt * (kh[0] * mh[1] * mh[2] + mh[0] * kh[1] * mh[2]
                                        + mh[0] * mh[1] * kh[2])
    err = torch.max(torch.abs(y.double() - lam * x.double())).item()
    M, K = orc.bspline_kernels(n, h)
    absW = np.sum(np.abs(M)) ** 3 + dt * 3 * np.sum(np.abs(K)) * np.sum(np.abs(M)) ** 2
    assert err <= 1e-5 * absW        # (|A| |x|)_i <= sum |W| for |x| <= 1
    del y
    modes = inputs.random_sine_modes(3, 64, 16)
    x = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float32)
    y = H.op_apply(x)
    rng = np.random.default_rng(0)
    pts = list(rng.integers(0, N ** 3, size=2500))
    for (k, j, i) in [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 5), (N - 1, 0, N - 2)]:
        pts.append((k * N + j) * N + i)
    for _ in range(496):
        c = rng.integers(0, N, size=3)
        c[rng.integers(0, 3)] = rng.choice([0, 1, 2, N - 3, N - 2, N - 1])
        pts.append((int(c[0]) * N + int(c[1])) * N + int(c[2]))
    pts = np.array(pts, dtype=np.int64)
    xh = x.cpu().numpy()
    p = orc.Problem(N, N, N, n, h, dt=dt)
    ref = orc.op_points(p, xh, pts)
    got = y.reshape(-1)[torch.from_numpy(pts).cuda()].double().cpu().numpy()
    bound = 1e-5 * absW * np.max(np.abs(xh))
    assert np.max(np.abs(got - ref)) <= bound


def test_full_size_928_heat_step_ir_closed_form(api):
    """928^3, 64 seeded sine modes, dt = 5e-4, the workload's 20 implicit Euler steps with FP32
    sweeps and FP64 refinement; each mode must decay by exactly its discrete factor g_k^20."""
    N, n, dt, tol, K = 928, 3, 5e-4, 1e-8, 20
    h = 1 / (N + 1)
    modes = inputs.random_sine_modes(3, 64, 16)
    u = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64)
    H = api.Handle(N, N, N, n, h, dt, precision="f32_ir")
    rep = H.heat_step(u, None, K, tol=tol)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol
    me, ke = exact_kernels(n)
    decayed = []
    for kv, a in modes:
        mh = [h * symbol(me, math.pi * k * h) for k in kv]
        kh = [symbol(ke, math.pi * k * h) / h for k in kv]
        M3 = mh[0] * mh[1] * mh[2]
        lam = M3 + dt * (kh[0] * mh[1] * mh[2] + mh[0] * kh[1] * mh[2] + mh[0] * mh[1] * kh[2])
        decayed.append((kv, a * (M3 / lam) ** K))
    want = inputs.sine_mode_field(N, N, N, decayed, device="cuda", dtype=torch.float64)
    err = (torch.linalg.vector_norm(u - want) / torch.linalg.vector_norm(want)).item()
    kappa = box_kappa(N, N, N, n, (h, h, h), dt)
    assert err <= K * kappa * tol, err


@pytest.mark.parametrize("precision", ["f64", "f32_ir", "f32"])
@pytest.mark.parametrize("pinned", [True, False])
def test_heat_step_host_buffers(api, orc, precision, pinned):
    """heat_step_host: the same step as heat_step on device vectors, from and back into host
    buffers (pinned or pageable), with a source term; the copies' device times are reported."""
    N, n, dt = (40, 28, 19), 3, 2e-3
    hs = tuple(1 / (k + 1) for k in N)
    H = api.Handle(*N, n, hs, dt, precision=precision)
    dt_t = torch.float32 if precision == "f32" else torch.float64
    u0 = inputs.random_field((N[2], N[1], N[0]), 21).to(dt_t)
    q = inputs.random_field((N[2], N[1], N[0]), 22).to(dt_t)
    ud = u0.cuda()
    rep_d = H.heat_step(ud, q.cuda(), 2, tol=1e-10)
    uh = u0.clone().pin_memory() if pinned else u0.clone()
    qh = q.clone().pin_memory() if pinned else q.clone()
    rep_h = H.heat_step_host(uh, qh, 2, tol=1e-10)
    assert rep_h["status"] == rep_d["status"] == 0
    # the same kernels on the same data; the dynamic item queue of the two-block CG kernel sums
    # the dot products in a run-dependent order, so the two solves may differ in the last bits
    assert abs(rep_h["iterations"] - rep_d["iterations"]) <= 2
    rel = (torch.linalg.vector_norm((uh - ud.cpu()).double()) / torch.linalg.vector_norm(ud.cpu().double())).item()
    assert rel <= (1e-4 if precision == "f32" else 1e-9), rel
    assert rep_h["h2d_ms"] > 0 and rep_h["d2h_ms"] > 0 and rep_h["elapsed_ms"] >= rep_h["h2d_ms"]
    with pytest.raises(ValueError):
        H.heat_step_host(ud, None, 1)                     # device tensors are not host buffers
