"""z-slab split on one GPU: several slabs of one grid in one process, halo planes moved by device
copies, against the oracle on the whole grid (FP64 parity at 1e-12).

- bsk_slab_apply: each slab's A x from its halo-extended planes equals the oracle's A x on the
  whole grid, planes z_off .. z_off + nz - 1. Halo planes beyond the global faces hold NaN, so
  a kernel that read them (instead of reflecting about the global face) would fail. Rows of
  16-byte multiples take the TMA kernel (FP32 up to degree 5, FP64 up to degree 3), the others
  the general kernel; the cases cover both.
- the slab CG driver: x after k iterations equals the oracle's CG iterate x_k element by
  element, and the converged solution solves the whole-grid system.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _halo_of(x, z, nz, n):
    """Planes z - n .. z + nz + n - 1 of the global x, NaN beyond the global faces."""
    nzg = x.shape[0]
    out = np.full((nz + 2 * n,) + x.shape[1:], np.nan)
    for i, g in enumerate(range(z - n, z + nz + n)):
        if 0 <= g < nzg:
            out[i] = x[g]
    return out


@pytest.mark.parametrize("n,shape,parts,prec", [
    (3, (37, 29, 23), [(0, 8), (8, 8), (16, 7)], "f64"),
    (3, (33, 20, 9), [(0, 3), (3, 3), (6, 3)], "f64"),      # slabs as thin as the halo
    (1, (40, 17, 6), [(0, 1), (1, 4), (5, 1)], "f64"),
    (2, (64, 48, 21), [(0, 10), (10, 11)], "f64"),
    (4, (35, 26, 30), [(0, 13), (13, 17)], "f64"),
    (5, (24, 22, 25), [(0, 5), (5, 12), (17, 8)], "f64"),
    (3, (64, 40, 26), [(0, 13), (13, 13)], "f32"),
    (5, (72, 30, 23), [(0, 5), (5, 9), (14, 9)], "f32"),
    (3, (32, 20, 9), [(0, 3), (3, 3), (6, 3)], "f64"),
], ids=lambda v: str(v).replace(" ", ""))
def test_slab_apply_matches_oracle(orc, n, shape, parts, prec):
    from paper_1904_03057_gb300 import slab as sl
    nx, ny, nzg = shape
    h, dt = 1.0 / (nzg + 1), 0.03
    rng = np.random.default_rng(11 + n)
    x = rng.standard_normal((nzg, ny, nx))
    prob = orc.Problem(nx, ny, nzg, n, h, dt=dt)
    dtype = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yref = orc.op_stencil(prob, x)
    scale = orc.abs_op(prob, x)
    tol = 1e-12 if prec == "f64" else 2.0 ** -20
    for z, nz in parts:
        s = sl.SlabHandle(nx, ny, z, nz, nzg, n, h, dt, precision=prec)
        xh = torch.from_numpy(_halo_of(x, z, nz, n)).to(device="cuda", dtype=dtype).contiguous()
        y = s.apply(xh).double().cpu().numpy()
        s.close()
        err = np.abs(y - yref[z:z + nz]) / np.maximum(scale[z:z + nz], 1e-300)
        assert np.isfinite(y).all(), f"slab {z}: read a plane beyond a global face"
        assert err.max() <= tol, (z, nz, err.max())


def test_set_slab_rejects_bad_placement():
    from paper_1904_03057_gb300 import slab as sl
    from paper_1904_03057_gb300 import _native
    with pytest.raises(_native.BskError):
        sl.SlabHandle(16, 16, 10, 8, 17, 3, 0.1)        # planes 10..17 of 17
    with pytest.raises(ValueError):
        sl.SlabHandle(16, 16, 0, 8, 17, 3, 0.1, precision="f32_ir")


def _split_cg(orc, shape, n, parts, iters=None, tol=1e-13):
    from paper_1904_03057_gb300 import slab as sl
    nx, ny, nzg = shape
    h, dt = 1.0 / (nzg + 1), 0.05
    rng = np.random.default_rng(5)
    b = rng.standard_normal((nzg, ny, nx))
    slabs = [sl.SlabHandle(nx, ny, z, nz, nzg, n, h, dt) for z, nz in parts]
    ex = sl.Exchange(0, None)
    bs = [torch.from_numpy(b[z:z + nz].copy()).cuda() for z, nz in parts]
    xs = [torch.zeros_like(t) for t in bs]
    rep = sl.cg_solve(slabs, ex, bs, xs, tol=tol if iters is None else 0.0,
                      max_iter=1000 if iters is None else iters, check_every=4)
    x = np.concatenate([t.cpu().numpy() for t in xs])
    for s in slabs:
        s.close()
    return orc.Problem(nx, ny, nzg, n, h, dt=dt), b, x, rep


@pytest.mark.parametrize("shape,parts", [((41, 30, 23), [(0, 12), (12, 11)]),
                                         ((41, 30, 23), [(0, 9), (9, 3), (12, 11)]),
                                         ((40, 30, 23), [(0, 12), (12, 11)])],
                         ids=["two-slabs", "three-slabs-thin-middle", "two-slabs-tma-rows"])
def test_slab_cg_iterates_match_oracle(orc, shape, parts):
    n, k = 3, 8
    prob, b, x, rep = _split_cg(orc, shape, n, parts, iters=k)
    assert rep["status"] == 1 and rep["iterations"] == k
    xr, it, _, st = orc.cg(prob, b, tol=0.0, max_iter=k)
    assert it == k
    # x_k of the same recurrence, summed in another order: FP64 rounding differences only
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()


def test_slab_cg_converges_to_the_whole_grid_solution(orc):
    prob, b, x, rep = _split_cg(orc, (50, 37, 29), 3, [(0, 15), (15, 14)])
    assert rep["status"] == 0
    res = b - orc.op_stencil(prob, x)
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(b)
    xr, it, rel, st = orc.cg(prob, b, tol=1e-13, max_iter=1000)
    assert abs(rep["iterations"] - it) <= 1
    assert np.linalg.norm(x - xr) <= 1e-11 * np.linalg.norm(xr)
