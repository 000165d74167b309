"""GB300-native tensor B-spline heat-equation solver (arXiv:1904.03057, hot path).

The CUDA library (``csrc/`` -> ``_build/libbsk.so``, C ABI in ``include/bsk.h``) applies the
implicit-Euler heat operator matrix-free and solves with device-resident conjugate gradients.
``api`` exposes the same entry points on torch CUDA tensors; ``inputs`` draws the seeded
synthetic workloads.
"""
from .api import (F32, F32_IR, F64, Handle, bsk_create, bspline_kernels, cg_solve, heat_step,
                  mass_apply, op_apply)

__all__ = ["F32", "F32_IR", "F64", "Handle", "bsk_create", "bspline_kernels", "cg_solve",
           "heat_step", "mass_apply", "op_apply"]
