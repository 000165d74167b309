"""Seeded synthetic inputs for the heat-equation workloads.

This module only draws problem data: node masks of spheres, sampled Gaussian sources, sums of
sine modes, random fields and batch problem lists. It holds none of the method's arithmetic (no
B-spline kernels, no operator, no solver), so both the CUDA path and the CPU oracle take their
inputs from here.

Node positions follow the grid convention of the library: an axis of N unknowns has step
h = 1/(N+1) (unless given) and nodes at x_i = i h, i = 1..N; arrays are laid out [nz][ny][nx].
Large fields are built with torch (on any device) through separable products, so a 928^3 field
is generated on the GPU in well under a second.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


def node_coords(N: int, h: float | None = None, device="cpu", dtype=torch.float64):
    h = 1.0 / (N + 1) if h is None else h
    return torch.arange(1, N + 1, device=device, dtype=dtype) * h


def sphere_mask(nx, ny, nz, center=(0.5, 0.5, 0.5), radius=0.45, h=None, device="cpu"):
    """uint8 node mask: 1 where |x_i - center| <= radius (closed ball)."""
    return union_of_spheres_mask(nx, ny, nz, [center], [radius], h=h, device=device)


def union_of_spheres_mask(nx, ny, nz, centers, radii, h=None, device="cpu"):
    hs = _steps(nx, ny, nz, h)
    xs = node_coords(nx, hs[0], device)
    ys = node_coords(ny, hs[1], device)
    zs = node_coords(nz, hs[2], device)
    m = torch.zeros((nz, ny, nx), dtype=torch.bool, device=device)
    for (cx, cy, cz), r in zip(centers, radii):
        d2 = ((zs - cz) ** 2)[:, None, None] + ((ys - cy) ** 2)[None, :, None] + \
             ((xs - cx) ** 2)[None, None, :]
        m |= d2 <= r * r
    return m.to(torch.uint8)


def random_spheres(seed: int, count: int = 40, rmin: float = 0.05, rmax: float = 0.2):
    """count spheres, radius ~ U[rmin, rmax], centre ~ U[r, 1-r]^3 (inside the unit cube)."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(rmin, rmax, size=count)
    centers = [tuple(rng.uniform(r, 1.0 - r, size=3)) for r in radii]
    return centers, [float(r) for r in radii]


def gaussian_centers(seed: int, count: int, lo: float = 0.2, hi: float = 0.8):
    rng = np.random.default_rng(seed)
    return [tuple(c) for c in rng.uniform(lo, hi, size=(count, 3))]


def gaussian_source(nx, ny, nz, centers, sigma=0.03, h=None, mask=None, device="cpu",
                    dtype=torch.float64):
    """Samples g(x_i) of g(x) = sum_s exp(-|x - c_s|^2 / (2 sigma^2)) at the nodes (zero on
    masked-out nodes). Each Gaussian is a separable product, so the sum costs one outer product
    per source."""
    hs = _steps(nx, ny, nz, h)
    xs = node_coords(nx, hs[0], device, dtype)
    ys = node_coords(ny, hs[1], device, dtype)
    zs = node_coords(nz, hs[2], device, dtype)
    g = torch.zeros((nz, ny, nx), dtype=dtype, device=device)
    s2 = 2.0 * sigma * sigma
    for (cx, cy, cz) in centers:
        gx = torch.exp(-(xs - cx) ** 2 / s2)
        gy = torch.exp(-(ys - cy) ** 2 / s2)
        gz = torch.exp(-(zs - cz) ** 2 / s2)
        g += gz[:, None, None] * (gy[:, None] * gx[None, :])[None, :, :]
    if mask is not None:
        g = g * mask.to(device=device, dtype=dtype)
    return g


def random_sine_modes(seed: int, count: int = 64, kmax: int = 16):
    """count distinct wave-vectors (k1, k2, k3) in {1..kmax}^3 with amplitudes
    N(0,1) / (k1^2 + k2^2 + k3^2)."""
    rng = np.random.default_rng(seed)
    picked = set()
    modes = []
    while len(modes) < count:
        k = tuple(int(v) for v in rng.integers(1, kmax + 1, size=3))
        if k in picked:
            continue
        picked.add(k)
        a = float(rng.standard_normal()) / float(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
        modes.append((k, a))
    return modes


def sine_mode_field(nx, ny, nz, modes, h=None, device="cpu", dtype=torch.float64):
    """F[k, j, i] = sum_m a_m sin(pi k1 x_i) sin(pi k2 y_j) sin(pi k3 z_k). Built plane by plane
    as a rank-len(modes) product, which is exact separable arithmetic on the samples."""
    hs = _steps(nx, ny, nz, h)
    xs = node_coords(nx, hs[0], device, dtype)
    ys = node_coords(ny, hs[1], device, dtype)
    zs = node_coords(nz, hs[2], device, dtype)
    kx = torch.tensor([m[0][0] for m in modes], device=device, dtype=dtype)
    ky = torch.tensor([m[0][1] for m in modes], device=device, dtype=dtype)
    kz = torch.tensor([m[0][2] for m in modes], device=device, dtype=dtype)
    a = torch.tensor([m[1] for m in modes], device=device, dtype=dtype)
    Sx = torch.sin(torch.pi * xs[:, None] * kx[None, :])   # [nx, M]
    Sy = torch.sin(torch.pi * ys[:, None] * ky[None, :])   # [ny, M]
    Sz = torch.sin(torch.pi * zs[:, None] * kz[None, :])   # [nz, M]
    out = torch.empty((nz, ny, nx), dtype=dtype, device=device)
    for k in range(nz):
        out[k] = (Sy * (Sz[k] * a)[None, :]) @ Sx.T
    return out


def random_field(shape, seed: int, device="cpu", dtype=torch.float64, mask=None):
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn(shape, generator=g, dtype=torch.float64).to(device=device, dtype=dtype)
    if mask is not None:
        x = x * mask.to(device=device, dtype=dtype)
    return x


def inclusion_coefficients(nx, ny, nz, seed: int, count: int = 8, base: float = 1.0,
                           lo: float = 0.2, hi: float = 5.0, h=None, device="cpu",
                           dtype=torch.float64):
    """Nodal coefficient field on the N + 2 nodes 0..N+1 of each axis (faces included, node e at
    position e h), shape (nz+2, ny+2, nx+2): the value base, overwritten inside `count` random
    balls (radius ~ U[0.1, 0.25], centre ~ U[0, 1]^3) by a value ~ log-uniform on [lo, hi] --
    a piecewise-constant material map such as tissue conductivities, with contrast up to hi/lo."""
    hs = _steps(nx, ny, nz, h)
    rng = np.random.default_rng(seed)
    axes = [torch.arange(0, N + 2, device=device, dtype=torch.float64) * hh
            for N, hh in zip((nx, ny, nz), hs)]
    out = torch.full((nz + 2, ny + 2, nx + 2), float(base), dtype=torch.float64, device=device)
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, size=3)
        r = rng.uniform(0.1, 0.25)
        v = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        d2 = ((axes[2] - c[2]) ** 2)[:, None, None] + ((axes[1] - c[1]) ** 2)[None, :, None] + \
             ((axes[0] - c[0]) ** 2)[None, None, :]
        out[d2 <= r * r] = v
    return out.to(dtype)


@dataclass
class BatchProblem:
    nx: int
    ny: int
    nz: int
    degree: int
    h: float
    centers: list = field(default_factory=list)


def batch_problems(seed: int = 4, count: int = 64, lo: int = 48, hi: int = 160,
                   degrees=(2, 3, 4, 5), sources: int = 8):
    """count independent box problems: dims ~ U{lo..hi} per axis, degree drawn from degrees,
    isotropic step h = 1/(max dim + 1), sources Gaussian centres ~ U[0.2, 0.8] scaled to the box."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        deg = int(rng.choice(degrees))
        h = 1.0 / (max(nx, ny, nz) + 1)
        ext = np.array([(nx + 1) * h, (ny + 1) * h, (nz + 1) * h])
        cs = [tuple(c) for c in rng.uniform(0.2, 0.8, size=(sources, 3)) * ext]
        out.append(BatchProblem(nx, ny, nz, deg, h, cs))
    return out


def _steps(nx, ny, nz, h):
    if h is None:
        return (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
    if np.isscalar(h):
        return (float(h),) * 3
    return tuple(float(v) for v in h)
