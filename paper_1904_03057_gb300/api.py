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

F64, F32, F32_IR = 0, 1, 2
_PREC = {"f64": F64, "f32": F32, "f32_ir": F32_IR, F64: F64, F32: F32, F32_IR: F32_IR}

OK, NOT_CONVERGED, STALLED = 0, 1, 2
KERNEL_OP, KERNEL_CG_FUSED, KERNEL_CG_UPDATE, KERNEL_RES64 = 0, 1, 2, 3
EINVAL, ECUDA, ENOMEM, ETIMEOUT, EBREAKDOWN = -1, -2, -3, -4, -5


def bspline_kernels(n: int, h: float):
    """(mass, stiff): the 2n+1 tap Galerkin kernels of degree-n B-splines on a grid of step h."""
    L = _native.load()
    m = np.zeros(2 * n + 1)
    k = np.zeros(2 * n + 1)
    _native.check(L.bspline_kernels(int(n), float(h), m.ctypes.data, k.ctypes.data))
    return m, k


def _opts(tol=None, max_iter=None, check_every=None, stall_window=None, inner_tol=None,
          max_outer=None, time_limit_s=None):
    o = _native.CgOpts()
    o.tol = float(tol or 0.0)
    o.max_iter = int(max_iter or 0)
    o.check_every = int(check_every or 0)
    o.stall_window = int(stall_window or 0)
    o.inner_tol = float(inner_tol or 0.0)
    o.max_outer = int(max_outer or 0)
    o.time_limit_s = float(time_limit_s or 0.0)
    return o


def _report(rep: _native.CgReport) -> dict:
    return {"status": rep.status, "iterations": rep.iterations,
            "outer_iterations": rep.outer_iterations, "rel_residual": rep.rel_residual,
            "elapsed_ms": rep.elapsed_ms, "kernel_launches": rep.kernel_launches}


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
        self.dtype = torch.float32 if self.precision == F32 else torch.float64
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

    def time_kernel(self, kernel: int, reps: int = 10) -> float:
        """Mean device time (ms) of one launch of a library kernel (bsk_time_kernel)."""
        out = ctypes.c_double(0.0)
        _native.check(self._lib.bsk_time_kernel(self._ptr, int(kernel), int(reps),
                                                ctypes.byref(out)))
        return out.value

    def norm2(self, x: torch.Tensor) -> float:
        out = ctypes.c_double(0.0)
        _native.check(self._lib.bsk_norm2(self._ptr, self._vec(x, "x"), ctypes.byref(out)))
        return out.value


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
