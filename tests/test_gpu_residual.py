"""The true residual of iterative refinement, r = b - A x: the double-float TMA kernel (FP32
pipes) and the FP64 kernels against the FP64 oracle, element by element, and the refinement run
with either."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api as a
    return a


CASES = [((30, 50, 68), 3, False), ((24, 37, 130), 3, True), ((20, 26, 64), 2, False),
         ((17, 30, 66), 1, True), ((12, 9, 22), 3, False), ((40, 30, 70), 4, False)]


@pytest.mark.parametrize("shape,n,masked", CASES)
@pytest.mark.parametrize("fp64", [False, True])
def test_residual_matches_oracle(api, shape, n, masked, fp64):
    """Both kernels agree with the oracle to 1e-12 of the |A||x| + |b| scale (the FP64 bar);
    shape (40, 30, 70) at degree 4 and the odd-row grid take the general FP64 kernel."""
    nz, ny, nx = shape
    h = 1.0 / (max(shape) + 1)
    dt = 7e-4
    rng = np.random.default_rng(hash((shape, n, masked)) % (1 << 31))
    mask = (rng.random(shape) < 0.6).astype(np.uint8) if masked else None
    x = rng.standard_normal(shape) * (mask if masked else 1.0)
    # b close to A x, as in refinement: the residual is a small difference of large terms
    P = oracle.Problem(nx, ny, nz, n, h, dt=dt, mask=mask)
    ax = oracle.op_stencil(P, x)
    b = ax + 1e-6 * np.abs(ax).max() * rng.standard_normal(shape)
    if masked:
        b_in = b.copy()
        b_in[mask == 0] = 123.0          # ignored
        b = b * mask
    else:
        b_in = b
    r_ref = b - ax
    scale = np.max(oracle.abs_op(P, np.abs(x)) + np.abs(b))
    H = api.Handle(nx, ny, nz, n, h, dt, precision="f32_ir",
                   mask=torch.from_numpy(mask).cuda() if masked else None)
    r, rr, bb = H.residual(torch.from_numpy(b_in).cuda(), torch.from_numpy(x).cuda(), fp64=fp64)
    r = r.cpu().numpy()
    err = np.max(np.abs(r - r_ref)) / scale
    assert err <= 1e-12, err
    assert abs(rr - np.sum(r_ref ** 2)) <= 1e-9 * np.sum(r_ref ** 2)
    assert abs(bb - np.sum(b ** 2)) <= 1e-12 * np.sum(b ** 2)
    if masked:
        assert np.all(r[mask == 0] == 0)
    H.close()


def test_refinement_with_either_residual(api):
    """cg_solve (BSK_F32_IR) reaches the tolerance with the double-float and with the FP64
    residual, with the same refinement steps and solutions equal to the tolerance's scale."""
    N = 64
    h = 1.0 / (N + 1)
    rng = np.random.default_rng(5)
    b = torch.from_numpy(rng.standard_normal((N, N, N)) * h ** 3).cuda()
    H = api.Handle(N, N, N, 3, h, 1e-3, precision="f32_ir")
    xs = []
    reps = []
    for fp64 in (False, True):
        x = torch.zeros_like(b)
        reps.append(H.cg_solve(b, x, tol=1e-10, residual_fp64=fp64))
        xs.append(x)
    assert all(r["status"] == 0 and r["rel_residual"] <= 1e-10 for r in reps), reps
    assert reps[0]["outer_iterations"] == reps[1]["outer_iterations"]
    d = (torch.linalg.vector_norm(xs[0] - xs[1]) / torch.linalg.vector_norm(xs[1])).item()
    assert d <= 1e-8, d
    H.close()


def test_sparse_mask_skips_empty_bricks(api):
    """A mask whose active nodes fill a few of the 64 x 24 tiles: the TMA kernels skip the
    empty (tile, z-chunk) items. Residual parity and zeros off the mask, and CG solves (FP64 and
    FP32 with refinement) that the oracle confirms."""
    from paper_1904_03057_gb300 import inputs
    nx, ny, nz, n, dt = 200, 80, 64, 3, 1e-3
    h = 1.0 / (nx + 1)
    mask = inputs.union_of_spheres_mask(nx, ny, nz, [(0.2, 0.15, 0.15), (0.7, 0.25, 0.2)], [0.06, 0.08],
                                        h=h)
    m = mask.numpy()
    tiles_active = sum(int(m[:, ty * 24:(ty + 1) * 24, tx * 64:(tx + 1) * 64].any())
                       for ty in range((ny + 23) // 24) for tx in range((nx + 63) // 64))
    assert 0 < tiles_active < 8            # most of the 16 tiles are empty
    rng = np.random.default_rng(3)
    x = rng.standard_normal((nz, ny, nx)) * m
    b = rng.standard_normal((nz, ny, nx)) * m * h ** 3
    P = oracle.Problem(nx, ny, nz, n, h, dt=dt, mask=m)
    r_ref = b - oracle.op_stencil(P, x)
    scale = np.max(oracle.abs_op(P, np.abs(x)) + np.abs(b))
    H = api.Handle(nx, ny, nz, n, h, dt, mask=mask.cuda(), precision="f32_ir")
    r, rr, bb = H.residual(torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda())
    r = r.cpu().numpy()
    assert np.max(np.abs(r - r_ref)) <= 1e-12 * scale
    assert np.all(r[m == 0] == 0)
    tol = 1e-9
    for prec in ("f32_ir", "f64"):
        Hs = api.Handle(nx, ny, nz, n, h, dt, mask=mask.cuda(), precision=prec)
        u = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
        rep = Hs.cg_solve(torch.from_numpy(b).cuda(), u, tol=tol)
        assert rep["status"] == 0, rep
        un = u.cpu().numpy()
        assert np.all(un[m == 0] == 0)
        res = b - oracle.op_stencil(P, un)
        assert np.linalg.norm(res) <= 1.5 * tol * np.linalg.norm(b), prec
        Hs.close()
    H.close()
