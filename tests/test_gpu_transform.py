"""B-spline transforms at the nodes on the GPU (bsk_transform) against the oracle's direct and
indirect transforms (section 2.3): every degree, anisotropic grids, both precisions, the
round trip, and the mask being ignored."""
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


CASES = [((10, 9, 12), 1), ((13, 11, 17), 2), ((20, 18, 40), 3), ((9, 14, 11), 4), ((12, 10, 16), 5),
         ((33, 29, 68), 3)]


@pytest.mark.parametrize("shape,n", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_transforms_match_oracle(api, shape, n, prec):
    nz, ny, nx = shape
    hs = (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
    P = oracle.Problem(nx, ny, nz, n, *hs)
    rng = np.random.default_rng(n * 100 + nx)
    c = rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    u_ref = oracle.indirect_transform(P, c)
    c_ref = oracle.direct_transform(P, f)
    dtype = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-13 if prec == "f64" else 2e-6
    H = api.Handle(nx, ny, nz, n, hs, 1e-3, precision=prec)
    u = H.to_samples(torch.from_numpy(c).to("cuda", dtype)).double().cpu().numpy()
    assert np.max(np.abs(u - u_ref)) <= tol * np.max(np.abs(u_ref)) * 4
    cg = H.to_coeffs(torch.from_numpy(f).to("cuda", dtype)).double().cpu().numpy()
    # the direct transform amplifies by at most 1 / (smallest symbol value) < 8 for n <= 5
    assert np.max(np.abs(cg - c_ref)) <= tol * 8 * np.max(np.abs(c_ref)) * 4
    H.close()


def test_round_trip_and_mask_ignored(api):
    from paper_1904_03057_gb300 import inputs
    N, n = 48, 3
    h = 1.0 / (N + 1)
    mask = inputs.sphere_mask(N, N, N, radius=0.3, h=h).cuda()
    modes = inputs.random_sine_modes(7, 16, 8)
    f = inputs.sine_mode_field(N, N, N, modes, device="cuda", dtype=torch.float64)
    Hm = api.Handle(N, N, N, n, h, 1e-3, mask=mask, precision="f32_ir")
    H = api.Handle(N, N, N, n, h, 1e-3, precision="f32_ir")
    c1 = Hm.to_coeffs(f)
    c2 = H.to_coeffs(f)
    assert torch.equal(c1, c2)                        # the mask does not enter the transforms
    back = H.to_samples(c2)
    assert (torch.max(torch.abs(back - f)) / torch.max(torch.abs(f))).item() <= 1e-13
    with pytest.raises(Exception):
        H._lib and api._native.check(H._lib.bsk_transform(H._ptr, 7, f.data_ptr(), c1.data_ptr()))
    Hm.close()
    H.close()
