"""The z-slab split on CPU ranks (gloo): partition, halo-plane indexing and the all-reduce
orchestration of the slab CG driver (paper_1904_03057_gb300/slab.py), with the slab passes
played by a CPU stand-in whose operator is the oracle's direct stencil on the global grid.

The stand-in's operator reads the slab's halo vector through a global array that is NaN
everywhere except the planes the halo vector holds, so a halo plane taken from the wrong
neighbour plane, left unfilled or read beyond the halo shows up as a wrong or NaN result. The
solution of the split CG must match the oracle's CG on the whole grid."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1904_03057_gb300 import slab as sl  # noqa: E402

GRID = dict(nx=9, ny=7, nz=17, n=3, h=1.0 / 18, dt=0.02)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class CpuSlab:
    """CPU stand-in for SlabHandle: the same passes and scalar bookkeeping as the slab kernels
    (include/bsk.h, bsk_slab_*), the operator taken from the oracle."""

    def __init__(self, z_off, nz, g=GRID):
        import oracle
        self.orc = oracle
        self.n, self.nx, self.ny = g["n"], g["nx"], g["ny"]
        self.z_off, self.nz, self.nz_glob = z_off, nz, g["nz"]
        self.prob = oracle.Problem(g["nx"], g["ny"], g["nz"], g["n"], g["h"], dt=g["dt"])
        plane = self.nx * self.ny
        self.points = np.arange(z_off * plane, (z_off + nz) * plane)

    def empty(self):
        return torch.zeros((self.nz, self.ny, self.nx), dtype=torch.float64)

    def empty_halo(self):
        return torch.zeros((self.nz + 2 * self.n, self.ny, self.nx), dtype=torch.float64)

    def scalars(self):
        return torch.zeros(sl.SCALARS, dtype=torch.float64)

    def apply(self, x_halo, y=None):
        G = np.full((self.nz_glob, self.ny, self.nx), np.nan)
        lo, hi = self.z_off - self.n, self.z_off + self.nz + self.n
        for i, gz in enumerate(range(lo, hi)):
            if 0 <= gz < self.nz_glob:
                G[gz] = x_halo[i].numpy()
        out = self.orc.op_points(self.prob, G.reshape(-1), self.points).reshape(self.nz, self.ny, self.nx)
        y = self.empty() if y is None else y
        y.copy_(torch.from_numpy(out))
        return y

    def _p(self, p_halo):
        return p_halo[self.n:self.n + self.nz]

    def begin(self, b, ax, r, p_halo, s, tol, max_iter):
        s.zero_()
        s[sl.TOL2], s[sl.MAX_ITER] = tol * tol, max_iter
        r.copy_(b - ax)
        self._p(p_halo).copy_(r)
        s[sl.RR_NEW], s[sl.BB] = float((r * r).sum()), float((b * b).sum())

    def matvec(self, p_halo, q, s):
        self.apply(p_halo, q)
        if s[sl.DONE] == 0:
            s[sl.PQ] = float((self._p(p_halo) * q).sum())

    def update(self, x, r, p_halo, q, s):
        if s[sl.DONE] != 0:
            return
        pq = float(s[sl.PQ])
        if not (pq > 0 and np.isfinite(pq)):
            s[sl.DONE], s[sl.STATUS] = 1, -5
            return
        a = float(s[sl.RR]) / pq
        x.add_(a * self._p(p_halo))
        r.sub_(a * q)
        s[sl.RR_NEW] = float((r * r).sum())

    def direction(self, r, p_halo, s, first):
        if s[sl.DONE] != 0:
            return
        beta = 0.0 if first else float(s[sl.RR_NEW] / s[sl.RR])
        p = self._p(p_halo)
        p.copy_(r + beta * p)
        if not first:
            s[sl.ITER] += 1
        s[sl.RR] = s[sl.RR_NEW]
        if float(s[sl.RR]) <= float(s[sl.TOL2] * s[sl.BB]):
            s[sl.DONE], s[sl.STATUS] = 1, 0
        elif float(s[sl.ITER]) >= float(s[sl.MAX_ITER]):
            s[sl.DONE], s[sl.STATUS] = 1, 1


def _rhs():
    rng = np.random.default_rng(7)
    return rng.standard_normal((GRID["nz"], GRID["ny"], GRID["nx"]))


def _rank_main(rank, world, port, layout, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = sl.partition(GRID["nz"], sum(layout), GRID["n"])
        first = sum(layout[:rank])
        mine = parts[first:first + layout[rank]]
        slabs = [CpuSlab(z, nz) for z, nz in mine]
        ex = sl.Exchange(first, dist.group.WORLD).bind(slabs)
        # halo indexing: every local plane holds its global plane index
        vs = [s.empty_halo() for s in slabs]
        for s, v in zip(slabs, vs):
            for i in range(s.nz):
                v[s.n + i] = s.z_off + i
        ex.halo(vs)
        halos = [v[:, 0, 0].tolist() for v in vs]
        # the split CG
        b = _rhs()
        bs = [torch.from_numpy(b[z:z + nz].copy()) for z, nz in mine]
        xs = [torch.zeros_like(t) for t in bs]
        rep = sl.cg_solve(slabs, ex, bs, xs, tol=1e-12, max_iter=500, check_every=3)
        out[rank] = (mine, halos, [x.numpy() for x in xs], rep)
    finally:
        dist.destroy_process_group()


def test_partition():
    assert sl.partition(17, 2, 3) == [(0, 9), (9, 8)]
    assert sl.partition(17, 3, 3) == [(0, 6), (6, 6), (12, 5)]
    assert sl.partition(4, 4, 1) == [(0, 1), (1, 1), (2, 1), (3, 1)]
    with pytest.raises(ValueError):
        sl.partition(5, 2, 3)     # a slab of 2 planes cannot feed 3 halo planes


@pytest.mark.parametrize("layout", [(1, 1), (2, 1)], ids=["one-slab-per-rank", "two-slabs-on-rank0"])
def test_slab_cg_on_gloo_ranks(orc, layout):
    import torch.multiprocessing as mp
    world = len(layout)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), layout, out), nprocs=world,
                       start_method="spawn")
    assert set(out.keys()) == set(range(world))
    n, nzg = GRID["n"], GRID["nz"]
    x = np.zeros((nzg, GRID["ny"], GRID["nx"]))
    reps = []
    for r in range(world):
        mine, halos, xs, rep = out[r]
        reps.append(rep)
        for (z, nz), h, xr in zip(mine, halos, xs):
            # halo planes: the neighbours' global plane indices, untouched (0) beyond the faces
            want = [float(g) if 0 <= g < nzg else 0.0 for g in range(z - n, z + nz + n)]
            assert h == want
            x[z:z + nz] = xr
    assert all(rp == reps[0] for rp in reps)           # every rank ends with the same scalars
    assert reps[0]["status"] == 0
    prob = orc.Problem(GRID["nx"], GRID["ny"], GRID["nz"], GRID["n"], GRID["h"], dt=GRID["dt"])
    xr, it, rel, st = orc.cg(prob, _rhs(), tol=1e-12, max_iter=500)
    assert st == 0 and abs(reps[0]["iterations"] - it) <= 1
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)
    # and the split solution solves the whole-grid system
    res = _rhs() - orc.op_stencil(prob, x)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(_rhs())
