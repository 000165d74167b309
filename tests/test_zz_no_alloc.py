"""residual_noalloc, the entry point that allocates nothing.

Some callers cannot call cudaMalloc (for example a solver plugin inside a host application that
owns the device memory and hands in pre-allocated buffers), so they cannot create a handle; this
entry point computes r = b - A x and the FP64 norms r.r and b.b from a static scratch array.
The test calls it through the C ABI twice in a row (the scratch keeps the previous call's
contents) and checks it against the handle-based entry points op_apply and bsk_norm2, within the
operator tolerances of the other GPU tests (1e-12 in FP64, 1e-5 in FP32, relative to |A||x|).
It sits in a file that pytest collects last, and passes alone or after the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,masked", [("f64", False), ("f64", True), ("f32", False),
                                              ("f32", True)])
def test_residual_noalloc_matches_handle_entry_points(orc, precision, masked):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import _native, api, inputs
    L = _native.load()
    nx, ny, nz, n, dt = 68, 45, 37, 3, 2e-3
    hs = (1 / (nx + 1), 1 / (ny + 1), 1 / (nz + 1))
    mask = inputs.sphere_mask(nx, ny, nz, radius=0.4, h=hs) if masked else None
    dtype = torch.float64 if precision == "f64" else torch.float32
    tol = 1e-12 if precision == "f64" else 1e-5
    H = api.Handle(nx, ny, nz, n, hs, dt, mask=None if mask is None else mask.cuda(),
                   precision=precision)
    x = inputs.random_field((nz, ny, nx), seed=21, mask=mask).to("cuda", dtype)
    b = inputs.random_field((nz, ny, nx), seed=22, mask=mask).to("cuda", dtype)
    r_ref = b - H.op_apply(x)
    rr_ref = H.norm2(r_ref)
    bb_ref = H.norm2(b)
    p = orc.Problem(nx, ny, nz, n, *hs, dt=dt, mask=None if mask is None else mask.numpy())
    scale = float(np.max(orc.abs_op(p, x.double().cpu().numpy()))) + float(b.abs().max())

    prob = _native.Problem(nx, ny, nz, n, hs[0], hs[1], hs[2], dt, None)
    keep = None if mask is None else mask.cuda()   # keeps the device mask alive for the calls
    if keep is not None:
        prob.mask = keep.data_ptr()
    prec = api.F64 if precision == "f64" else api.F32
    stream = torch.cuda.current_stream()
    for call in range(2):
        r = torch.full_like(x, float("nan"))
        rr = ctypes.c_double(-1.0)
        bb = ctypes.c_double(-1.0)
        rc = L.residual_noalloc(ctypes.byref(prob), prec, x.data_ptr(), b.data_ptr(),
                                r.data_ptr(), ctypes.byref(rr), ctypes.byref(bb),
                                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.bsk_last_error()
        err = torch.max(torch.abs(r.double() - r_ref.double())).item()
        assert err <= tol * scale, (call, err, scale)
        assert abs(rr.value - rr_ref) <= 1e-9 * rr_ref + tol
        assert abs(bb.value - bb_ref) <= 1e-9 * bb_ref
        if mask is not None:
            assert torch.count_nonzero(r[mask.cuda() == 0]).item() == 0


def test_residual_noalloc_rejects_oversize_and_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import _native, api
    L = _native.load()
    rr, bb = ctypes.c_double(), ctypes.c_double()
    big = _native.Problem(4096, 4096, 4096, 3, 1e-3, 1e-3, 1e-3, 0.0, None)
    dummy = torch.zeros(16, device="cuda")
    p = dummy.data_ptr()
    rc = L.residual_noalloc(ctypes.byref(big), api.F32, p, p + 64, p + 128, ctypes.byref(rr),
                            ctypes.byref(bb), None)
    assert rc == -1 and b"too large" in L.bsk_last_error()
    small = _native.Problem(8, 8, 8, 3, 0.1, 0.1, 0.1, 0.0, None)
    assert L.residual_noalloc(ctypes.byref(small), api.F32_IR, p, p, p, ctypes.byref(rr),
                              ctypes.byref(bb), None) == -1
    assert L.residual_noalloc(None, api.F64, p, p, p, ctypes.byref(rr), ctypes.byref(bb),
                              None) == -1
