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
    # the oracle's residual of the same inputs (FP64, the definition of b - A x)
    xin = x.double().cpu().numpy()
    r_orc = b.double().cpu().numpy() - orc.op_separable(p, xin)
    if mask is not None:
        r_orc = r_orc * mask.numpy()
    rs = [torch.full_like(x, float("nan")) for _ in range(2)]   # allocated before the calls
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        r = rs[call]
        rr = ctypes.c_double(-1.0)
        bb = ctypes.c_double(-1.0)
        # free device memory right around the call: nothing else runs in between (the checks
        # below allocate through torch's caching allocator)
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        rc = L.residual_noalloc(ctypes.byref(prob), prec, x.data_ptr(), b.data_ptr(),
                                r.data_ptr(), ctypes.byref(rr), ctypes.byref(bb),
                                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.bsk_last_error()
        torch.cuda.synchronize()
        free.append((before, torch.cuda.mem_get_info()[0]))
        err = torch.max(torch.abs(r.double() - r_ref.double())).item()
        assert err <= tol * scale, (call, err, scale)
        err_orc = float(np.max(np.abs(r.double().cpu().numpy() - r_orc)))
        assert err_orc <= tol * scale, (call, err_orc, scale)
        assert abs(rr.value - rr_ref) <= 1e-9 * rr_ref + tol
        assert abs(rr.value - float(np.sum(r_orc * r_orc))) <= 1e-9 * rr.value + tol * scale * np.sqrt(r_orc.size)
        assert abs(bb.value - bb_ref) <= 1e-9 * bb_ref
        if mask is not None:
            assert torch.count_nonzero(r[mask.cuda() == 0]).item() == 0
    # the second call (module loaded, scratch address known) took no device memory
    assert free[1][1] == free[1][0], free


def test_residual_noalloc_rejects_oversize_and_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import _native, api
    L = _native.load()
    rr, bb = ctypes.c_double(), ctypes.c_double()
    dummy = torch.zeros(16, device="cuda")
    p = dummy.data_ptr()
    # the bound is ceil(nx/32) * ceil(ny/16) <= 16384 blocks of the general kernel, any nz:
    # 4096 x 2049 x 3 is just over it, 4096 x 2048 x 3 at it
    for big in (_native.Problem(4096, 4096, 4096, 3, 1e-3, 1e-3, 1e-3, 0.0, None),
                _native.Problem(4096, 2049, 3, 3, 1e-3, 1e-3, 1e-3, 0.0, None)):
        rc = L.residual_noalloc(ctypes.byref(big), api.F32, p, p + 64, p + 128, ctypes.byref(rr),
                                ctypes.byref(bb), None)
        assert rc == -1 and b"too large" in L.bsk_last_error()
    edge = _native.Problem(4096, 2048, 3, 3, 1e-3, 1e-3, 1e-3, 1e-4, None)
    x = torch.ones((3, 2048, 4096), device="cuda")
    b = torch.ones_like(x)
    r = torch.empty_like(x)
    rc = L.residual_noalloc(ctypes.byref(edge), api.F32, x.data_ptr(), b.data_ptr(), r.data_ptr(),
                            ctypes.byref(rr), ctypes.byref(bb), None)
    assert rc == 0, L.bsk_last_error()
    assert bb.value == float(x.numel()) and rr.value >= 0.0
    del x, b, r
    # a call on a stream that is capturing a graph is refused and leaves the capture intact
    small = _native.Problem(8, 8, 8, 3, 0.1, 0.1, 0.1, 0.0, None)
    xs = torch.ones((8, 8, 8), device="cuda")
    bs = torch.ones_like(xs)
    rs_ = torch.empty_like(xs)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        xs.add_(0.0)
        rc = L.residual_noalloc(ctypes.byref(small), api.F32, xs.data_ptr(), bs.data_ptr(), rs_.data_ptr(),
                                ctypes.byref(rr), ctypes.byref(bb), ctypes.c_void_p(side.cuda_stream))
    assert rc == -1 and b"capturing" in L.bsk_last_error()
    g.replay()
    torch.cuda.synchronize()
    small = _native.Problem(8, 8, 8, 3, 0.1, 0.1, 0.1, 0.0, None)
    assert L.residual_noalloc(ctypes.byref(small), api.F32_IR, p, p, p, ctypes.byref(rr),
                              ctypes.byref(bb), None) == -1
    assert L.residual_noalloc(None, api.F64, p, p, p, ctypes.byref(rr), ctypes.byref(bb),
                              None) == -1
