"""Batched solver (bsk_batch_*): many independent box problems of mixed sizes and degrees in one
persistent launch per degree, vs one-by-one solves and the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1904_03057_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

SMALL = [  # nx, ny, nz, degree -- ragged rows (nx not a multiple of 4), tiny and multi-tile grids
    (21, 17, 13, 2), (37, 29, 23, 3), (70, 30, 26, 4), (9, 11, 7, 5), (48, 50, 31, 3),
    (5, 6, 5, 5), (66, 26, 40, 2),
]


class P:
    def __init__(self, nx, ny, nz, degree):
        self.nx, self.ny, self.nz, self.degree = nx, ny, nz, degree
        self.h = 1.0 / (max(nx, ny, nz) + 1)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api as a
    return a


def test_batch_cg_matches_single_solves_and_oracle(api, orc):
    dt, tol = 2e-3, 1e-10
    probs = [P(*t) for t in SMALL]
    B = api.BatchHandle(probs, dt)
    bs, xs = [], []
    for i, p in enumerate(probs):
        b = inputs.random_field((p.nz, p.ny, p.nx), seed=100 + i).cuda()
        bs.append(b)
        xs.append(torch.zeros_like(b))
    bs[3] = torch.zeros_like(bs[3])          # one trivial problem: x = 0, no iterations
    reps = B.cg_solve(bs, xs, tol=tol)
    for i, (p, r) in enumerate(zip(probs, reps)):
        assert r["status"] == 0, (i, r)
        assert r["rel_residual"] <= tol
        if i == 3:
            assert torch.count_nonzero(xs[i]).item() == 0 and r["iterations"] == 0
            continue
        H = api.Handle(p.nx, p.ny, p.nz, p.degree, p.h, dt, precision="f32_ir")
        x1 = torch.zeros_like(bs[i])
        H.cg_solve(bs[i], x1, tol=tol)
        q = orc.Problem(p.nx, p.ny, p.nz, p.degree, p.h, dt=dt)
        xb = xs[i].cpu().numpy()
        bn = bs[i].cpu().numpy()
        true_rel = np.linalg.norm(bn - orc.op_separable(q, xb)) / np.linalg.norm(bn)
        assert true_rel <= 1.5 * tol
        d = (torch.linalg.vector_norm(xs[i] - x1) / torch.linalg.vector_norm(x1)).item()
        assert d <= 1e-6, (i, d)


def test_batch_heat_step_matches_single_handles(api):
    dt, tol, K = 1e-3, 1e-9, 2
    probs = [P(*t) for t in SMALL[:5]]
    B = api.BatchHandle(probs, dt)
    us, qs, ref = [], [], []
    for i, p in enumerate(probs):
        cs = inputs.gaussian_centers(40 + i, 4)
        q = inputs.gaussian_source(p.nx, p.ny, p.nz, cs, 0.05, h=p.h).cuda()
        u0 = inputs.random_field((p.nz, p.ny, p.nx), seed=7 + i).cuda() * 0.1
        us.append(u0.clone())
        qs.append(q)
        H = api.Handle(p.nx, p.ny, p.nz, p.degree, p.h, dt, precision="f64")
        u1 = u0.clone()
        H.heat_step(u1, q, K, tol=tol)
        ref.append(u1)
    reps = B.heat_step(us, qs, K, tol=tol)
    for i in range(len(probs)):
        assert reps[i]["status"] == 0
        d = (torch.linalg.vector_norm(us[i] - ref[i]) / torch.linalg.vector_norm(ref[i])).item()
        assert d <= 1e-6, (i, d)


def test_batch_autotune_then_solve(api, tmp_path):
    dt, tol = 1e-3, 1e-8
    probs = [P(*t) for t in SMALL]
    B = api.BatchHandle(probs, dt)
    res = api.autotune_cached(B, probs, str(tmp_path / "tune.json"))
    assert res["check_every"] >= 2 and not res["cached"]
    assert sorted(g["degree"] for g in res["groups"]) == [2, 3, 4, 5]
    for g in res["groups"]:
        assert g["nzc"] in (1, 2, 3, 4, 6, 8) and g["ms"] > 0
        assert g["tile"] in ([64, 16], [64, 24], [64, 32] if g["degree"] <= 4 else [64, 24])
    assert abs(sum(g["ms"] for g in res["groups"]) - res["ms_per_iteration"]) <= 1e-9
    res2 = api.autotune_cached(B, probs, str(tmp_path / "tune.json"))
    assert res2["cached"] and res2["groups"] == res["groups"]
    assert [(g["degree"], g["tile"], g["nzc"]) for g in B.groups()] == \
        [(g["degree"], g["tile"], g["nzc"]) for g in res["groups"]]
    bs = [inputs.random_field((p.nz, p.ny, p.nx), seed=300 + i).cuda() for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    reps = B.cg_solve(bs, xs, tol=tol)
    assert all(r["status"] == 0 and r["rel_residual"] <= tol for r in reps)


@pytest.mark.parametrize("rows,nzc", [(16, 1), (16, 3), (24, 2), (32, 1), (32, 4)])
def test_batch_tile_shapes_agree(api, orc, rows, nzc):
    """Each tile shape (64 x 16, 24, 32; 32 for degrees <= 4) and z-chunking solves the mixed
    batch to the same tolerance, with the oracle's true residual, the same iteration counts as
    the 64 x 24 tiles up to rounding, and the same solutions."""
    dt, tol = 2e-3, 1e-10
    probs = [P(*t) for t in SMALL]
    bs = [inputs.random_field((p.nz, p.ny, p.nx), seed=500 + i).cuda() for i, p in enumerate(probs)]

    def solve(r, c):
        B = api.BatchHandle(probs, dt)
        B.configure([{"degree": d, "tile": [64, r if (r < 32 or d <= 4) else 24], "nzc": c}
                     for d in sorted({p.degree for p in probs})], 16)
        xs = [torch.zeros_like(b) for b in bs]
        reps = B.cg_solve(bs, xs, tol=tol)
        groups = B.groups()
        B.close()
        return xs, reps, groups

    x0, r0, _ = solve(24, 1)
    xs, reps, groups = solve(rows, nzc)
    for g in groups:
        assert g["tile"][1] == (rows if (rows < 32 or g["degree"] <= 4) else 24) and g["nzc"] == nzc
    for i, (p, r) in enumerate(zip(probs, reps)):
        assert r["status"] == 0 and r["rel_residual"] <= tol, (i, r)
        q = orc.Problem(p.nx, p.ny, p.nz, p.degree, p.h, dt=dt)
        bn, xn = bs[i].cpu().numpy(), xs[i].cpu().numpy()
        assert np.linalg.norm(bn - orc.op_separable(q, xn)) <= 1.5 * tol * np.linalg.norm(bn)
        d = (torch.linalg.vector_norm(xs[i] - x0[i]) / torch.linalg.vector_norm(x0[i])).item()
        assert d <= 1e-8, (i, d)
        # Iteration counts follow the rounding (the dot products are summed in another order)
        # only mildly while FP32 CG keeps its directions conjugate. Where it needs more
        # iterations than the box has unknowns (the 5 x 6 x 5 quintic box: 150 unknowns, about
        # 570 iterations) orthogonality is lost and the count depends on rounding; it is not compared.
        if r0[i]["iterations"] < p.nx * p.ny * p.nz:
            assert abs(r["iterations"] - r0[i]["iterations"]) <= max(2, 0.05 * r0[i]["iterations"]), (i, r, r0[i])


def test_batch_configure_rejects_missing_tile(api):
    B = api.BatchHandle([P(*t) for t in SMALL], 1e-3)
    from paper_1904_03057_gb300 import _native
    with pytest.raises(_native.BskError):
        B.configure([{"degree": 5, "tile": [64, 32], "nzc": 1}], 16)   # no 64 x 32 tile at degree 5
    with pytest.raises(_native.BskError):
        B.configure([{"degree": 1, "tile": [64, 24], "nzc": 1}], 16)   # no problem of degree 1
    B.close()


def test_batch_64_boxes_one_step(api):
    """64 problems, dims U{48..160} per axis, degrees {2,3,4,5}, 8 Gaussian sources
    each, dt = 1e-3; one implicit Euler step of the whole batch to a 1e-8 true residual."""
    dt, tol = 1e-3, 1e-8
    specs = inputs.batch_problems(seed=4)
    B = api.BatchHandle(specs, dt)
    us, qs = [], []
    for s in specs:
        us.append(torch.zeros((s.nz, s.ny, s.nx), dtype=torch.float64, device="cuda"))
        qs.append(inputs.gaussian_source(s.nx, s.ny, s.nz, s.centers, 0.03, h=s.h, device="cuda"))
    reps = B.heat_step(us, qs, 1, tol=tol)
    assert all(r["status"] == 0 and r["rel_residual"] <= tol for r in reps)
    # spot checks against one-by-one solves
    for i in (0, 17, 63):
        s = specs[i]
        H = api.Handle(s.nx, s.ny, s.nz, s.degree, s.h, dt, precision="f32_ir")
        u = torch.zeros_like(us[i])
        H.heat_step(u, qs[i], 1, tol=tol)
        d = (torch.linalg.vector_norm(u - us[i]) / torch.linalg.vector_norm(u)).item()
        assert d <= 1e-5, (i, d)
