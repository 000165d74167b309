"""z-slab split of one grid across devices (section 3 of arXiv:1904.03057 distributes the
unknowns of one problem over several GPUs; here each device holds a contiguous range of
z-planes).

The operator of Eq. tensForm couples a plane to the n planes on each side (degree n), so each
slab keeps its search direction p with n halo planes below and above the local ones. One CG
iteration (section 2.5) on the slabs is

    exchange the halo planes of p         (device copies between the slabs of this process,
                                           send/recv to the neighbouring ranks)
    q = A p, local p.q                    bsk_slab_cg_matvec   -> all-reduce of p.q
    x += alpha p, r -= alpha q, local r.r bsk_slab_cg_update   -> all-reduce of r.r
    p = r + beta p, convergence test      bsk_slab_cg_direction

The passes are CUDA kernels behind the C ABI (include/bsk.h, bsk_slab_*); this module only
places the slabs, moves halo planes and sums the scalars between the passes. The scalars sit in
a small device array per slab, so an NCCL all-reduce acts on it in place, and the host reads it
only every `check_every` iterations (passes queued past convergence change nothing).

A process may hold several consecutive slabs (the test runs two slabs of one grid on one GPU
this way); with a torch.distributed group, rank k holds the k-th block of slabs.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import torch

from . import _native
from .api import Handle, _PREC

# Layout of the scalar array (BSK_SLAB_* in bsk.h).
PQ, RR_NEW, BB, RR, TOL2, MAX_ITER, ITER, DONE, STATUS = range(9)
SCALARS = 16


def partition(nz_glob: int, parts: int, degree: int) -> List[Tuple[int, int]]:
    """(z_off, nz) of each of `parts` consecutive slabs of a grid of nz_glob planes, as even as
    possible. Every slab needs at least `degree` planes, so that its halo planes come from its
    two neighbours only."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    base, extra = divmod(int(nz_glob), int(parts))
    if base < max(int(degree), 1):
        raise ValueError(f"{nz_glob} planes cannot give {parts} slabs of at least {degree} planes")
    out, z = [], 0
    for k in range(parts):
        nz = base + (1 if k < extra else 0)
        out.append((z, nz))
        z += nz
    return out


class SlabHandle:
    """One slab on this process's GPU: a handle for its local planes, placed in the global grid
    (bsk_create + bsk_set_slab), with the slab entry points."""

    def __init__(self, nx: int, ny: int, z_off: int, nz: int, nz_glob: int, degree: int, h,
                 dt: float = 0.0, precision="f64", stream: Optional[torch.cuda.Stream] = None):
        if _PREC[precision] not in (0, 1):
            raise ValueError("slab handles take precision 'f64' or 'f32'")
        self.handle = Handle(nx, ny, nz, degree, h, dt, precision=precision, stream=stream)
        self._lib = self.handle._lib
        self._ptr = self.handle._ptr
        self.n = int(degree)
        self.z_off, self.nz, self.nz_glob = int(z_off), int(nz), int(nz_glob)
        self.nx, self.ny = int(nx), int(ny)
        self.dtype = self.handle.dtype
        self.device = torch.device("cuda", torch.cuda.current_device())
        _native.check(self._lib.bsk_set_slab(self._ptr, self.z_off, self.nz_glob))

    def empty(self) -> torch.Tensor:
        return self.handle.empty()

    def empty_halo(self) -> torch.Tensor:
        """A zeroed (nz + 2n, ny, nx) vector: n halo planes, the local planes, n halo planes."""
        return torch.zeros((self.nz + 2 * self.n, self.ny, self.nx), dtype=self.dtype, device=self.device)

    def scalars(self) -> torch.Tensor:
        return torch.zeros(SCALARS, dtype=torch.float64, device=self.device)

    def _halo(self, t: torch.Tensor, name: str) -> int:
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()
                and tuple(t.shape) == (self.nz + 2 * self.n, self.ny, self.nx)):
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor of shape "
                             f"{(self.nz + 2 * self.n, self.ny, self.nx)}")
        return t.data_ptr()

    def _s(self, s: torch.Tensor) -> int:
        if not (s.is_cuda and s.dtype == torch.float64 and s.is_contiguous() and s.numel() >= SCALARS):
            raise ValueError(f"s must be a contiguous CUDA float64 tensor of {SCALARS} elements")
        return s.data_ptr()

    def apply(self, x_halo: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = self.empty() if y is None else y
        _native.check(self._lib.bsk_slab_apply(self._ptr, self._halo(x_halo, "x_halo"),
                                               self.handle._vec(y, "y")))
        return y

    def begin(self, b, ax, r, p_halo, s, tol: float, max_iter: int):
        v = self.handle._vec
        _native.check(self._lib.bsk_slab_cg_begin(self._ptr, v(b, "b"), v(ax, "ax"), v(r, "r"),
                                                  self._halo(p_halo, "p_halo"), self._s(s),
                                                  float(tol), int(max_iter)))

    def matvec(self, p_halo, q, s):
        _native.check(self._lib.bsk_slab_cg_matvec(self._ptr, self._halo(p_halo, "p_halo"),
                                                   self.handle._vec(q, "q"), self._s(s)))

    def update(self, x, r, p_halo, q, s):
        v = self.handle._vec
        _native.check(self._lib.bsk_slab_cg_update(self._ptr, v(x, "x"), v(r, "r"),
                                                   self._halo(p_halo, "p_halo"), v(q, "q"), self._s(s)))

    def direction(self, r, p_halo, s, first: bool):
        _native.check(self._lib.bsk_slab_cg_direction(self._ptr, self.handle._vec(r, "r"),
                                                      self._halo(p_halo, "p_halo"), self._s(s),
                                                      int(bool(first))))

    def close(self):
        self.handle.close()


class Exchange:
    """Halo exchange and scalar all-reduce over all slabs of one grid.

    This process holds consecutive slabs, the first of them global slab `first`; `group` (a
    torch.distributed process group, or None for a single process) connects the ranks, each
    holding a consecutive block of slabs. bind() records the local slab objects (anything with
    attributes n, nz and a scalars() method); the tensors handed to halo() and allreduce() live
    on one device per process (CUDA tensors with NCCL, CPU tensors with gloo)."""

    def __init__(self, first: int = 0, group=None):
        self.first, self.group = int(first), group
        self.dist = None
        if group is not None:
            import torch.distributed as dist
            self.dist = dist

    def bind(self, slabs: Sequence) -> "Exchange":
        """Records the local slabs and learns (one all-gather) which rank holds each slab."""
        self.slabs = list(slabs)
        self.local = range(self.first, self.first + len(self.slabs))
        self.owner = {g: None for g in self.local}
        if self.dist is not None:
            dev = self.slabs[0].scalars().device
            rank, world = self.dist.get_rank(self.group), self.dist.get_world_size(self.group)
            mine = torch.tensor([self.first, len(self.slabs)], dtype=torch.int64, device=dev)
            every = [torch.zeros(2, dtype=torch.int64, device=dev) for _ in range(world)]
            self.dist.all_gather(every, mine, group=self.group)
            self.owner = {}
            for k, t in enumerate(every):
                f, m = (int(v) for v in t.cpu())
                for g in range(f, f + m):
                    if g in self.owner:
                        raise ValueError(f"slab {g} is held by two ranks")
                    self.owner[g] = None if k == rank else k
            if sorted(self.owner) != list(range(len(self.owner))):
                raise ValueError("the ranks' slabs do not cover 0 .. nslabs - 1")
        self.total = len(self.owner)
        return self

    # -- scalars ---------------------------------------------------------------------------
    def allreduce(self, ss: Sequence[torch.Tensor], start: int, count: int) -> None:
        """Sums entries start .. start + count - 1 of the local slabs' scalar arrays over all
        slabs of the grid (the local ones in order, then across ranks) and writes the total back
        into each local array."""
        tot = ss[0][start:start + count].clone()
        for s in ss[1:]:
            tot += s[start:start + count]
        if self.dist is not None:
            self.dist.all_reduce(tot, group=self.group)
        for s in ss:
            s[start:start + count].copy_(tot)

    # -- halo planes -----------------------------------------------------------------------
    def halo(self, vs: Sequence[torch.Tensor]) -> None:
        """Fills the halo planes of the local slabs' halo vectors vs (nz + 2n planes each) from
        the neighbouring slabs' local planes: the lower halo of slab g from the top n local
        planes of slab g - 1, the upper halo from the bottom n local planes of slab g + 1. Halo
        planes beyond the global faces are left as they are (odd reflection never reads them)."""
        reqs = []
        for i, (sl, v) in enumerate(zip(self.slabs, vs)):
            g, n, nz = self.first + i, sl.n, sl.nz
            below, above = v[0:n], v[n + nz:2 * n + nz]    # halo planes
            bottom, top = v[n:2 * n], v[nz:nz + n]           # local planes the neighbours need
            for nb, dst, mine in ((g - 1, below, bottom), (g + 1, above, top)):
                if nb < 0 or nb >= self.total:
                    continue
                if self.owner[nb] is None:                   # a slab of this process
                    j = nb - self.first
                    other, w = self.slabs[j], vs[j]
                    src = w[other.nz:other.nz + other.n] if nb < g else w[other.n:2 * other.n]
                    dst.copy_(src)
                else:
                    reqs.append(self.dist.isend(mine, self.owner[nb], group=self.group))
                    reqs.append(self.dist.irecv(dst, self.owner[nb], group=self.group))
        for r in reqs:
            r.wait()


def cg_solve(slabs: Sequence, ex: Exchange, bs: Sequence[torch.Tensor], xs: Sequence[torch.Tensor],
             tol: float = 1e-10, max_iter: int = 10000, check_every: int = 1) -> dict:
    """CG (section 2.5) for A x = b on a grid split into z-slabs. slabs / bs / xs: this process's
    slabs (SlabHandle) with their local planes of b and of the starting x (updated in place);
    ex: the Exchange bound to these slabs. Returns status (0 converged, 1 max_iter, -5
    breakdown), iterations and the relative residual sqrt(r.r / b.b) of the recurrence."""
    ex.bind(slabs)
    xh = [sl.empty_halo() for sl in slabs]
    for sl, x, v in zip(slabs, xs, xh):
        v[sl.n:sl.n + sl.nz].copy_(x)
    ex.halo(xh)
    ax = [sl.apply(v) for sl, v in zip(slabs, xh)]
    del xh
    r = [sl.empty() for sl in slabs]
    q = [sl.empty() for sl in slabs]
    p = [sl.empty_halo() for sl in slabs]
    s = [sl.scalars() for sl in slabs]
    for i, sl in enumerate(slabs):
        sl.begin(bs[i], ax[i], r[i], p[i], s[i], tol, max_iter)
    ex.allreduce(s, RR_NEW, 2)
    for i, sl in enumerate(slabs):
        sl.direction(r[i], p[i], s[i], True)
    check_every = max(int(check_every), 1)
    while True:
        head = s[0].cpu()
        if head[DONE] != 0:
            break
        for _ in range(check_every):
            ex.halo(p)
            for i, sl in enumerate(slabs):
                sl.matvec(p[i], q[i], s[i])
            ex.allreduce(s, PQ, 1)
            for i, sl in enumerate(slabs):
                sl.update(xs[i], r[i], p[i], q[i], s[i])
            ex.allreduce(s, RR_NEW, 1)
            for i, sl in enumerate(slabs):
                sl.direction(r[i], p[i], s[i], False)
    bb = float(head[BB])
    rel = math.sqrt(float(head[RR]) / bb) if bb > 0 else 0.0
    return {"status": int(head[STATUS]), "iterations": int(head[ITER]), "rel_residual": rel}
