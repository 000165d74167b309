"""BF16-storage operator variant (BSK_BF16S): parity with the oracle on BF16 inputs, and the
accuracy BF16 storage costs against the FP64 operator on the unrounded field."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api, inputs
    return api, inputs


@pytest.mark.parametrize("shape,n,masked", [((20, 17, 33), 3, False), ((16, 24, 40), 2, True),
                                            ((12, 13, 14), 5, False)])
def test_bf16s_op_apply_matches_oracle(mods, shape, n, masked):
    """y = A x on bfloat16 x: FP32 arithmetic, one rounding of y to bfloat16. Bound per element:
    half a BF16 ulp of y (at most 2^-8 |y|: 8 significant bits) plus FP32 rounding (1e-5 of the
    |A||x| scale)."""
    api, inputs = mods
    nz, ny, nx = shape
    h = 1.0 / (max(shape) + 1)
    dt = 1e-3
    rng = np.random.default_rng(7)
    x64 = rng.standard_normal(shape)
    mask = (rng.random(shape) < 0.7).astype(np.uint8) if masked else None
    xb = torch.from_numpy(x64).to(torch.bfloat16)
    xr = xb.double().numpy()                      # the values the GPU actually reads
    P = oracle.Problem(nx, ny, nz, n, h, dt=dt, mask=mask)
    yref = oracle.op_stencil(P, xr)
    scale = np.max(oracle.abs_op(P, np.abs(xr)))
    H = api.Handle(nx, ny, nz, n, h, dt, precision="bf16s",
                   mask=torch.from_numpy(mask).cuda() if masked else None)
    y = H.op_apply(xb.cuda().contiguous()).double().cpu().numpy()
    err = np.abs(y - yref)
    bound = 2.0 ** -8 * np.abs(yref) * (1 + 1e-3) + 1e-5 * scale
    assert np.all(err <= bound), float(np.max(err / bound))
    if masked:
        assert np.all(y[mask == 0] == 0)
    H.close()


def test_bf16s_storage_error_vs_fp64(mods):
    """What BF16 storage costs: y_bf16 = A round_bf16(x) (FP32 arithmetic, BF16 output) against
    the FP64 operator of the unrounded x, relative 2-norm error. A smooth field (sine modes) keeps
    about BF16 precision; the stiffness kernels' cancellation amplifies it for rough fields."""
    api, inputs = mods
    N = 64
    h = 1.0 / (N + 1)
    dt = 5e-4
    modes = inputs.random_sine_modes(3, 64, 16)
    u = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64)
    rough = inputs.random_field((N, N, N), seed=11, device="cuda")
    H64 = api.Handle(N, N, N, 3, h, dt, precision="f64")
    Hb = api.Handle(N, N, N, 3, h, dt, precision="bf16s")
    errs = {}
    for name, f in (("smooth", u), ("rough", rough)):
        y64 = H64.op_apply(f)
        yb = Hb.op_apply(f.to(torch.bfloat16).contiguous()).double()
        errs[name] = (torch.linalg.vector_norm(yb - y64) / torch.linalg.vector_norm(y64)).item()
    print("BF16-storage relative error:", errs)
    assert errs["smooth"] < 2e-2
    assert errs["smooth"] > 2.0 ** -12          # it is a real loss of precision, not FP32-exact
    assert errs["rough"] < 1.0
    H64.close()
    Hb.close()


def test_bf16s_rejects_solvers(mods):
    api, inputs = mods
    H = api.Handle(16, 16, 16, 3, 1.0 / 17, 1e-3, precision="bf16s")
    b = torch.zeros((16, 16, 16), dtype=torch.bfloat16, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(Exception):
        H.cg_solve(b, x)
    with pytest.raises(Exception):
        H.heat_step(x)
    with pytest.raises(Exception):
        H.time_kernel(api.KERNEL_OP)
    H.close()
