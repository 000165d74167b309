"""ctypes binding of libbsk.so (include/bsk.h). Argument marshalling only: every step of the
path runs in the library's CUDA kernels. The library is loaded on first use (built first if it
is missing or older than its sources) and any failure to build or load raises: there is no
fallback."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None


class Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("degree", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mask", ctypes.c_void_p),
    ]


class CgOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
        ("stall_window", ctypes.c_int), ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int), ("time_limit_s", ctypes.c_double),
        ("residual_fp64", ctypes.c_int),
    ]


class CgReport(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int),
        ("outer_iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
        ("elapsed_ms", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
        ("fallback_iter", ctypes.c_int), ("net_rejected", ctypes.c_int), ("iter_ms", ctypes.c_double),
        ("h2d_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double),
    ]


# exported symbols and their signatures: (restype, argtypes)
SIGNATURES = {
    "bspline_kernels": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "bsk_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "bsk_destroy": (None, [ctypes.c_void_p]),
    "bsk_set_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "op_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mass_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport)]),
    "heat_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport)]),
    "bsk_norm2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_double)]),
    "bsk_transform": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "bsk_set_coefficients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_set_boundary": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "bsk_set_preconditioner": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bsk_prolong": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_op_flops": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]),
    "bsk_time_kernel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]),
    "bsk_select_cg_kernel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "bsk_cg_kernel_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bsk_set_slab": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bsk_inverse_diagonal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "heat_step_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "fcg_record": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int)]),
    "bsk_slab_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_slab_cg_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "bsk_slab_cg_matvec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_slab_cg_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_slab_cg_direction": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int]),
    "residual_noalloc": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "bsk_batch_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "bsk_batch_destroy": (None, [ctypes.c_void_p]),
    "bsk_batch_cg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(CgOpts), ctypes.POINTER(CgReport)]),
    "bsk_batch_heat_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.POINTER(CgOpts),
                                           ctypes.POINTER(CgReport)]),
    "bsk_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]),
    "bsk_batch_groups": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_batch_configure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int]),
    "bsk_net_param_count": (ctypes.c_int, []),
    "bsk_net_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "bsk_net_destroy": (None, [ctypes.c_void_p]),
    "bsk_net_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_net_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bsk_net_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "bsk_net_set_activation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bsk_net_zero_grad": (ctypes.c_int, [ctypes.c_void_p]),
    "bsk_net_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_float]),
    "bsk_net_backward_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_float]),
    "bsk_net_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_float]),
    "bsk_net_read_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                         ctypes.c_void_p]),
    "fcg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.POINTER(CgOpts),
                                 ctypes.POINTER(CgReport)]),
    "bsk_last_error": (ctypes.c_char_p, []),
    "bsk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libbsk.so (building it first if needed and allowed). Raises on any failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class BskError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bsk status {code}: {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc < 0:
        L = load()
        raise BskError(rc, L.bsk_last_error().decode())
    return rc
