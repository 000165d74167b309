"""Python face of the C ABI (include/bsk.h): the same entry points, taking torch CUDA tensors.

Only argument marshalling happens here (shape/dtype/device checks, pointer and stream
extraction). PyTorch supplies device memory and streams; all arithmetic runs in libbsk.so.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _native

F64, F32, F32_IR, BF16S = 0, 1, 2, 3
_PREC = {"f64": F64, "f32": F32, "f32_ir": F32_IR, "bf16s": BF16S,
         F64: F64, F32: F32, F32_IR: F32_IR, BF16S: BF16S}

OK, NOT_CONVERGED, STALLED = 0, 1, 2
KERNEL_OP, KERNEL_CG_FUSED, KERNEL_CG_UPDATE, KERNEL_RES64, KERNEL_RES_DF = 0, 1, 2, 3, 4
CG_KERNEL_AUTO, CG_KERNEL_WS, CG_KERNEL_CLASSIC, CG_KERNEL_CURRENT = 0, 1, 2, 3
CG_KERNEL_WS_CHUNKED, CG_KERNEL_WS_COLUMNS = 4, 5
EINVAL, ECUDA, ENOMEM, ETIMEOUT, EBREAKDOWN = -1, -2, -3, -4, -5


def bspline_kernels(n: int, h: float):
    """(mass, stiff): the 2n+1 tap Galerkin kernels of degree-n B-splines on a grid of step h."""
    L = _native.load()
    m = np.zeros(2 * n + 1)
    k = np.zeros(2 * n + 1)
    _native.check(L.bspline_kernels(int(n), float(h), m.ctypes.data, k.ctypes.data))
    return m, k


def _opts(tol=None, max_iter=None, check_every=None, stall_window=None, inner_tol=None,
          max_outer=None, time_limit_s=None, residual_fp64=None):
    o = _native.CgOpts()
    o.tol = float(tol or 0.0)
    o.max_iter = int(max_iter or 0)
    o.check_every = int(check_every or 0)
    o.stall_window = int(stall_window or 0)
    o.inner_tol = float(inner_tol or 0.0)
    o.max_outer = int(max_outer or 0)
    o.time_limit_s = float(time_limit_s or 0.0)
    o.residual_fp64 = int(bool(residual_fp64))
    return o


def _report(rep: _native.CgReport) -> dict:
    return {"status": rep.status, "iterations": rep.iterations,
            "outer_iterations": rep.outer_iterations, "rel_residual": rep.rel_residual,
            "elapsed_ms": rep.elapsed_ms, "kernel_launches": rep.kernel_launches,
            "fallback_iter": rep.fallback_iter, "net_rejected": rep.net_rejected,
            "iter_ms": rep.iter_ms, "h2d_ms": rep.h2d_ms, "d2h_ms": rep.d2h_ms}


class Handle:
    """A solver handle for one box problem (bsk_create / bsk_destroy)."""

    def __init__(self, nx: int, ny: int, nz: int, degree: int, h, dt: float = 0.0,
                 mask: Optional[torch.Tensor] = None, precision="f64",
                 stream: Optional[torch.cuda.Stream] = None):
        self._lib = _native.load()
        self._ptr = ctypes.c_void_p(None)
        hx, hy, hz = (float(h),) * 3 if np.isscalar(h) else tuple(float(v) for v in h)
        self.shape = (int(nz), int(ny), int(nx))
        self.degree = int(degree)
        self.precision = _PREC[precision]
        self.dtype = {F32: torch.float32, BF16S: torch.bfloat16}.get(self.precision, torch.float64)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prob = _native.Problem(int(nx), int(ny), int(nz), int(degree), hx, hy, hz, float(dt), None)
        self._mask = None
        if mask is not None:
            if not (mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()
                    and tuple(mask.shape) == self.shape):
                raise ValueError("mask must be a contiguous CUDA uint8 tensor of shape (nz, ny, nx)")
            self._mask = mask
            prob.mask = mask.data_ptr()
        _native.check(self._lib.bsk_create(ctypes.byref(prob), self.precision,
                                           ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(self._ptr)))

    # -- helpers ---------------------------------------------------------------------------
    def _vec(self, t: torch.Tensor, name: str) -> int:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype:
            raise ValueError(f"{name} must have dtype {self.dtype}, got {t.dtype}")
        if not t.is_contiguous() or t.numel() != self.shape[0] * self.shape[1] * self.shape[2]:
            raise ValueError(f"{name} must be contiguous with {self.shape} elements")
        return t.data_ptr()

    def empty(self) -> torch.Tensor:
        return torch.empty(self.shape, dtype=self.dtype, device="cuda")

    def close(self):
        if self._ptr:
            self._lib.bsk_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points ----------------------------------------------------------------------
    def set_dt(self, dt: float):
        _native.check(self._lib.bsk_set_dt(self._ptr, float(dt)))

    def op_apply(self, x: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = self.empty() if y is None else y
        _native.check(self._lib.op_apply(self._ptr, self._vec(x, "x"), self._vec(y, "y")))
        return y

    def mass_apply(self, x: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = self.empty() if y is None else y
        _native.check(self._lib.mass_apply(self._ptr, self._vec(x, "x"), self._vec(y, "y")))
        return y

    def cg_solve(self, b: torch.Tensor, x: torch.Tensor, **opts) -> dict:
        o = _opts(**opts)
        rep = _native.CgReport()
        _native.check(self._lib.cg_solve(self._ptr, self._vec(b, "b"), self._vec(x, "x"),
                                         ctypes.byref(o), ctypes.byref(rep)))
        return _report(rep)

    def heat_step(self, u: torch.Tensor, q: Optional[torch.Tensor] = None, nsteps: int = 1,
                  **opts) -> dict:
        o = _opts(**opts)
        rep = _native.CgReport()
        qp = self._vec(q, "q") if q is not None else None
        _native.check(self._lib.heat_step(self._ptr, self._vec(u, "u"), qp, int(nsteps),
                                          ctypes.byref(o), ctypes.byref(rep)))
        return _report(rep)

    def heat_step_host(self, u: torch.Tensor, q: Optional[torch.Tensor] = None, nsteps: int = 1,
                       **opts) -> dict:
        """heat_step on HOST tensors (heat_step_host): u (and q) are copied to the device, stepped
        and u copied back, inside the library; pinned tensors copy at the link's speed."""
        def host(t, name):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() \
                    or t.numel() != self.shape[0] * self.shape[1] * self.shape[2]:
                raise ValueError(f"{name} must be a contiguous host tensor of dtype {self.dtype} with "
                                 f"{self.shape} elements")
            return t.data_ptr()
        o = _opts(**opts)
        rep = _native.CgReport()
        _native.check(self._lib.heat_step_host(self._ptr, host(u, "u"), None if q is None else host(q, "q"),
                                               int(nsteps), ctypes.byref(o), ctypes.byref(rep)))
        return _report(rep)

    def fcg_solve(self, b: torch.Tensor, x: torch.Tensor, net: Optional["Net"] = None,
                  **opts) -> dict:
        """Flexible CG with the learned preconditioner (net=None: no preconditioner) inside
        iterative refinement (BSK_F32_IR handles)."""
        o = _opts(**opts)
        rep = _native.CgReport()
        _native.check(self._lib.fcg_solve(self._ptr, net._ptr if net is not None else None,
                                          self._vec(b, "b"), self._vec(x, "x"), ctypes.byref(o),
                                          ctypes.byref(rep)))
        return _report(rep)

    def fcg_record(self, b: torch.Tensor, steps: int, net: Optional["Net"] = None):
        """The states of one inner flexible-CG solve from x = 0 (fcg_record): returns (r, d,
        bnorm) with r[k], d[k] the inner residual and iterate of A d = b / ||b|| before
        iteration k (float32, k < the number recorded) and bnorm = ||b||."""
        n = self.shape
        r = torch.empty((steps,) + n, dtype=torch.float32, device="cuda")
        d = torch.empty_like(r)
        bn, k = ctypes.c_double(0.0), ctypes.c_int(0)
        _native.check(self._lib.fcg_record(self._ptr, net._ptr if net is not None else None, self._vec(b, "b"),
                                           int(steps), r.data_ptr(), d.data_ptr(), ctypes.byref(bn),
                                           ctypes.byref(k)))
        return r[:k.value], d[:k.value], bn.value

    def time_kernel(self, kernel: int, reps: int = 10) -> float:
        """Mean device time (ms) of one launch of a library kernel (bsk_time_kernel)."""
        out = ctypes.c_double(0.0)
        _native.check(self._lib.bsk_time_kernel(self._ptr, int(kernel), int(reps),
                                                ctypes.byref(out)))
        return out.value

    def select_cg_kernel(self, request: str = "auto") -> str:
        """Kernel of the single-pass FP32 CG iteration (bsk_select_cg_kernel): "auto" times the
        candidates and keeps the fastest, "ws" (its z-chunking timed) / "classic" force a kernel,
        "ws_chunked" / "ws_columns" the warp-specialised pass with a fixed item plan, "current"
        only reports. Returns the kernel now in use."""
        req = {"auto": CG_KERNEL_AUTO, "ws": CG_KERNEL_WS, "classic": CG_KERNEL_CLASSIC,
               "current": CG_KERNEL_CURRENT, "ws_chunked": CG_KERNEL_WS_CHUNKED,
               "ws_columns": CG_KERNEL_WS_COLUMNS}[request]
        out = ctypes.c_int(0)
        _native.check(self._lib.bsk_select_cg_kernel(self._ptr, req, ctypes.byref(out)))
        return "ws" if out.value == CG_KERNEL_WS else "classic"

    def cg_kernel_config(self) -> dict:
        """The CG kernel in use and, for the warp-specialised pass, its z-chunk cap in planes."""
        k, c = ctypes.c_int(0), ctypes.c_int(0)
        _native.check(self._lib.bsk_cg_kernel_config(self._ptr, ctypes.byref(k), ctypes.byref(c)))
        return {"kernel": "ws" if k.value == CG_KERNEL_WS else "classic", "zchunk_planes": c.value}

    def norm2(self, x: torch.Tensor) -> float:
        out = ctypes.c_double(0.0)
        _native.check(self._lib.bsk_norm2(self._ptr, self._vec(x, "x"), ctypes.byref(out)))
        return out.value

    def to_samples(self, c: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Values at the grid nodes of the B-spline coefficients c (indirect transform)."""
        out = self.empty() if out is None else out
        _native.check(self._lib.bsk_transform(self._ptr, 0, self._vec(c, "c"), self._vec(out, "out")))
        return out

    def to_coeffs(self, f: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """B-spline coefficients interpolating the node values f (direct transform)."""
        out = self.empty() if out is None else out
        _native.check(self._lib.bsk_transform(self._ptr, 1, self._vec(f, "f"), self._vec(out, "out")))
        return out

    def residual(self, b: torch.Tensor, x: torch.Tensor, r: Optional[torch.Tensor] = None,
                 fp64: bool = False):
        """(r, ||r||^2, ||b||^2) with r = b - A x by the handle's true-residual kernel
        (bsk_residual)."""
        r = self.empty() if r is None else r
        rr, bb = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _native.check(self._lib.bsk_residual(self._ptr, self._vec(b, "b"), self._vec(x, "x"),
                                             self._vec(r, "r"), int(bool(fp64)), ctypes.byref(rr),
                                             ctypes.byref(bb)))
        return r, rr.value, bb.value

    @property
    def coef_shape(self):
        """Shape of a nodal coefficient field: the N + 2 nodes 0..N+1 of each axis."""
        return (self.shape[0] + 2, self.shape[1] + 2, self.shape[2] + 2)

    def set_coefficients(self, d: Optional[torch.Tensor] = None, m: Optional[torch.Tensor] = None):
        """Variable coefficients (bsk_set_coefficients): D = sum d beta and mu_a = sum m beta from
        float64 CUDA fields of shape coef_shape (None = 1 everywhere; both None = back to the
        constant-coefficient operator). The handle copies them."""
        ptrs = []
        for name, f in (("d", d), ("m", m)):
            if f is None:
                ptrs.append(None)
                continue
            if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == torch.float64
                    and f.is_contiguous() and tuple(f.shape) == self.coef_shape):
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape {self.coef_shape}")
            ptrs.append(f.data_ptr())
        _native.check(self._lib.bsk_set_coefficients(self._ptr, ptrs[0], ptrs[1]))

    def set_boundary(self, kind: str = "dirichlet", penalty: float = 0.0):
        """'dirichlet' (odd reflection) or 'robin' (untruncated basis with the boundary penalty
        term; the handle's dimensions are then the unknowns per axis, see robin_size)."""
        k = {"dirichlet": 0, "robin": 1}[kind]
        _native.check(self._lib.bsk_set_boundary(self._ptr, k, float(penalty)))

    def inverse_diagonal(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """1 / diag A per node (bsk_inverse_diagonal; needs set_preconditioner("jacobi"))."""
        out = self.empty() if out is None else out
        _native.check(self._lib.bsk_inverse_diagonal(self._ptr, self._vec(out, "out")))
        return out

    def set_preconditioner(self, kind: str = "none"):
        """'none' or 'jacobi' (Jacobi-preconditioned CG)."""
        k = {"none": 0, "jacobi": 1}[kind]
        _native.check(self._lib.bsk_set_preconditioner(self._ptr, k))

    def op_flops(self):
        """(algorithmic, executed) floating-point operations per node of one operator
        application (bsk_op_flops)."""
        a, e = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _native.check(self._lib.bsk_op_flops(self._ptr, ctypes.byref(a), ctypes.byref(e)))
        return a.value, e.value


def robin_size(degree: int, N: int) -> int:
    """Unknowns per axis of a Robin handle on a box of N interior nodes: N + 2 + 2 floor(n/2)."""
    return int(N) + 2 + 2 * (int(degree) // 2)


def prolong(fine: "Handle", coarse: "Handle", xc: torch.Tensor,
            xf: Optional[torch.Tensor] = None) -> torch.Tensor:
    """L2 projection of a coarse Robin expansion onto the fine Robin basis (bsk_prolong)."""
    xf = fine.empty() if xf is None else xf
    _native.check(fine._lib.bsk_prolong(fine._ptr, coarse._ptr, coarse._vec(xc, "xc"), fine._vec(xf, "xf")))
    return xf


class BatchHandle:
    """Many independent unmasked box problems solved together (bsk_batch_*). problems: a list of
    objects with nx, ny, nz, degree, h (scalar or 3-tuple); all share dt. Vectors are float64."""

    def __init__(self, problems, dt: float, stream: Optional[torch.cuda.Stream] = None):
        self._lib = _native.load()
        self._ptr = ctypes.c_void_p(None)
        self.count = len(problems)
        self.shapes = []
        arr = (_native.Problem * self.count)()
        for i, p in enumerate(problems):
            hs = (float(p.h),) * 3 if np.isscalar(p.h) else tuple(float(v) for v in p.h)
            arr[i] = _native.Problem(int(p.nx), int(p.ny), int(p.nz), int(p.degree), hs[0], hs[1],
                                     hs[2], float(dt), None)
            self.shapes.append((int(p.nz), int(p.ny), int(p.nx)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _native.check(self._lib.bsk_batch_create(arr, self.count, F32_IR,
                                                 ctypes.c_void_p(self.stream.cuda_stream),
                                                 ctypes.byref(self._ptr)))

    def _ptrs(self, vecs, name, allow_none=False):
        if vecs is None:
            return None
        if len(vecs) != self.count:
            raise ValueError(f"{name}: expected {self.count} vectors")
        out = (ctypes.c_void_p * self.count)()
        for i, (v, shp) in enumerate(zip(vecs, self.shapes)):
            if v is None and allow_none:
                out[i] = None
                continue
            if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64
                    and v.is_contiguous() and v.numel() == shp[0] * shp[1] * shp[2]):
                raise ValueError(f"{name}[{i}] must be a contiguous CUDA float64 tensor of {shp}")
            out[i] = v.data_ptr()
        return out

    def _reports(self, reps):
        return [_report(r) for r in reps]

    def cg_solve(self, bs, xs, **opts):
        o = _opts(**opts)
        reps = (_native.CgReport * self.count)()
        _native.check(self._lib.bsk_batch_cg_solve(self._ptr, self._ptrs(bs, "b"),
                                                   self._ptrs(xs, "x"), ctypes.byref(o), reps))
        return self._reports(reps)

    def heat_step(self, us, qs=None, nsteps: int = 1, **opts):
        o = _opts(**opts)
        reps = (_native.CgReport * self.count)()
        _native.check(self._lib.bsk_batch_heat_step(self._ptr, self._ptrs(us, "u"),
                                                    self._ptrs(qs, "q", allow_none=True),
                                                    int(nsteps), ctypes.byref(o), reps))
        return self._reports(reps)

    def autotune(self, reps: int = 3) -> dict:
        """Times every tile shape x z-chunking per degree group and keeps the fastest
        (bsk_batch_autotune). Returns the graph length, the ms of one batched iteration and,
        per group, the degree, tile [64, rows], z-chunks and ms."""
        ce, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        _native.check(self._lib.bsk_batch_autotune(self._ptr, int(reps), ctypes.byref(ce), ctypes.byref(ms)))
        return {"check_every": ce.value, "ms_per_iteration": ms.value, "groups": self.groups()}

    def groups(self) -> list:
        """Per degree group: degree, tile [columns, rows], z-chunks per problem, tuned ms per pass."""
        n = _native.check(self._lib.bsk_batch_groups(self._ptr, 0, None, None, None, None))
        deg, rows, nzc = (np.zeros(n, dtype=np.int32) for _ in range(3))
        ms = np.zeros(n)
        _native.check(self._lib.bsk_batch_groups(self._ptr, n, deg.ctypes.data, rows.ctypes.data,
                                                 nzc.ctypes.data, ms.ctypes.data))
        return [{"degree": int(d), "tile": [64, int(r)], "nzc": int(c), "ms": float(t)}
                for d, r, c, t in zip(deg, rows, nzc, ms)]

    def configure(self, groups, check_every: int):
        """Sets each group's tile and z-chunks (a list as returned by groups()) and the graph length."""
        for g in groups:
            _native.check(self._lib.bsk_batch_configure(self._ptr, int(g["degree"]), int(g["tile"][1]),
                                                        int(g["nzc"]), int(check_every)))

    def close(self):
        if self._ptr:
            self._lib.bsk_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The learned preconditioner network for one grid (bsk_net_*)."""

    def __init__(self, nx: int, ny: int, nz: int, stream: Optional[torch.cuda.Stream] = None,
                 activation: str = "relu"):
        self._lib = _native.load()
        self._ptr = ctypes.c_void_p(None)
        self.shape = (int(nz), int(ny), int(nx))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nparam = self._lib.bsk_net_param_count()
        _native.check(self._lib.bsk_net_create(int(nx), int(ny), int(nz),
                                               ctypes.c_void_p(self.stream.cuda_stream),
                                               ctypes.byref(self._ptr)))
        self.set_activation(activation)

    def set_activation(self, activation: str):
        """"relu" or "linear" (bsk_net_set_activation)."""
        act = {"relu": 0, "linear": 1}[activation]
        _native.check(self._lib.bsk_net_set_activation(self._ptr, act))
        self.activation = activation

    def _f32(self, t, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and tuple(t.shape) == self.shape):
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of {self.shape}")
        return t.data_ptr()

    @staticmethod
    def _mask(m):
        return None if m is None else m.data_ptr()

    def set_params(self, params: torch.Tensor):
        p = params.detach().to(torch.float32).contiguous()
        assert p.numel() == self.nparam
        _native.check(self._lib.bsk_net_set_params(self._ptr, p.data_ptr()))
        torch.cuda.current_stream().synchronize()

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.nparam, dtype=torch.float32)
        _native.check(self._lib.bsk_net_get_params(self._ptr, out.data_ptr()))
        return out

    def forward(self, r: torch.Tensor, mask=None, z: Optional[torch.Tensor] = None):
        z = torch.empty_like(r) if z is None else z
        _native.check(self._lib.bsk_net_forward(self._ptr, self._f32(r, "r"), self._mask(mask),
                                                self._f32(z, "z")))
        return z

    def zero_grad(self):
        _native.check(self._lib.bsk_net_zero_grad(self._ptr))

    def backward(self, r, e, mask=None, loss_weight=None):
        if loss_weight is None:
            active = r.numel() if mask is None else int(mask.sum().item())
            loss_weight = 2.0 / max(active, 1)
        _native.check(self._lib.bsk_net_backward(self._ptr, self._f32(r, "r"), self._f32(e, "e"),
                                                 self._mask(mask), float(loss_weight)))

    def backward_grad(self, r, dz, mask=None, scale: float = 1.0):
        """Parameter gradients for a caller-evaluated loss with output gradient dz."""
        _native.check(self._lib.bsk_net_backward_grad(self._ptr, self._f32(r, "r"), self._f32(dz, "dz"),
                                                      self._mask(mask), float(scale)))

    def adam(self, lr: float, grad_scale: float = 1.0):
        _native.check(self._lib.bsk_net_adam(self._ptr, float(lr), float(grad_scale)))

    def read(self, grads: bool = False):
        loss = ctypes.c_float(0.0)
        g = np.zeros(self.nparam, dtype=np.float32) if grads else None
        _native.check(self._lib.bsk_net_read_loss(self._ptr, ctypes.byref(loss),
                                                  g.ctypes.data if grads else None))
        return (loss.value, g) if grads else loss.value

    def close(self):
        if self._ptr:
            self._lib.bsk_net_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Version of the autotuner's search space; results tuned over another space are not reused.
AUTOTUNE_SPACE = "tiles64x16,24,32;nzc1,2,3,4,6,8"


def autotune_cached(batch: BatchHandle, key_problems, cache_path: str, reps: int = 3) -> dict:
    """Autotunes a batch once per (GPU, search space, problem list) and keeps the result -- the
    tile shape and z-chunks of each degree group, and the graph length -- in a JSON cache file."""
    import hashlib
    import json
    import os
    gpu = torch.cuda.get_device_name()
    desc = ";".join(f"{p.nx}x{p.ny}x{p.nz}n{p.degree}" for p in key_problems)
    key = f"{gpu}|f32|{AUTOTUNE_SPACE}|{hashlib.sha1(desc.encode()).hexdigest()}"
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        batch.configure(cache[key]["groups"], cache[key]["check_every"])
        return dict(cache[key], cached=True)
    res = batch.autotune(reps)
    cache[key] = res
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return dict(res, cached=False)


# Module-level forms with the C ABI's names.
def bsk_create(nx, ny, nz, degree, h, dt=0.0, mask=None, precision="f64", stream=None) -> Handle:
    return Handle(nx, ny, nz, degree, h, dt, mask, precision, stream)


def op_apply(handle: Handle, x, y=None):
    return handle.op_apply(x, y)


def mass_apply(handle: Handle, x, y=None):
    return handle.mass_apply(x, y)


def cg_solve(handle: Handle, b, x, **opts):
    return handle.cg_solve(b, x, **opts)


def heat_step(handle: Handle, u, q=None, nsteps=1, **opts):
    return handle.heat_step(u, q, nsteps, **opts)
