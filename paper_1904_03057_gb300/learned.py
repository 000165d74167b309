"""Training data and training loop of the learned preconditioner (orchestration: the network,
its gradients, Adam and the operator run in the library's CUDA kernels through the C ABI; the
loss bookkeeping and the data-generation iteration use torch vector arithmetic).

Training pairs come from the plain solver: for a random masked box problem A x = b, the solver
gives x* (tight tolerance) and, stopped after k iterations, x_k; the pair is the residual
r_k = b - A x_k and the error e_k = x* - x_k, scaled to the input r_k / ||r_k|| and the target
e_k (hx hy hz) / ||r_k|| (the network's output unit, see fcg_solve in include/bsk.h). Training
minimises the relative energy-norm error (EnergyLoss) and then adds, over a few rounds, the
residuals that flexible CG with the network itself produces (fcg_pairs, train_on_policy).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import api, inputs


@dataclass
class PairSet:
    r: torch.Tensor      # [count, nz, ny, nx] float32, unit norm each
    e: torch.Tensor      # [count, nz, ny, nx] float32, scaled error
    mask: torch.Tensor   # [count, nz, ny, nx] uint8
    shape: tuple
    h: float = 1.0 / 513
    dt: float = 1e-3
    degree: int = 3


def _random_crop_mask(n, rng, device):
    """Union of 2..6 spheres (radius 0.15..0.45 of the crop) inside an n^3 crop, or the whole
    crop one time in five; at least one node active."""
    if rng.random() < 0.2:
        return torch.ones((n, n, n), dtype=torch.uint8, device=device)
    k = int(rng.integers(2, 7))
    radii = rng.uniform(0.15, 0.45, size=k)
    centers = [tuple(rng.uniform(0.2, 0.8, size=3)) for _ in range(k)]
    m = inputs.union_of_spheres_mask(n, n, n, centers, list(radii), h=1.0 / (n + 1), device=device)
    if int(m.sum().item()) == 0:
        m[n // 2, n // 2, n // 2] = 1
    return m


@dataclass
class CropProblem:
    mask: torch.Tensor   # [n, n, n] uint8
    b: torch.Tensor      # [n, n, n] float64, zero off the mask
    xs: torch.Tensor     # [n, n, n] float64, the solution of A x = b (tight tolerance)


def make_problems(count: int, crop: int = 48, h: float = 1.0 / 513, dt: float = 1e-3, seed: int = 0,
                  degree: int = 3, device="cuda", signed: bool = True,
                  noise_fraction: float = 0.0, domain_mask=None) -> list:
    """`count` random masked crop^3 problems with their solutions. The right-hand side is a few
    Gaussian sources plus a little noise, or (a fraction noise_fraction of the problems) white
    noise, which gives residuals rich in high frequencies. With `signed` each source gets a random
    sign and amplitude, so that the network learns no sign bias (a preconditioner has to act on
    r and -r alike). With domain_mask (a [nz][ny][nx] uint8 tensor of the target domain) the
    masks are random crop^3 windows of it that contain active nodes, so that the network sees
    the geometry it will precondition; otherwise unions of random spheres inside the crop."""
    rng = np.random.default_rng(seed)
    n = crop
    out = []
    for _ in range(count):
        if domain_mask is not None:
            for _try in range(100):
                z0, y0, x0 = (int(rng.integers(0, d - n + 1)) for d in domain_mask.shape)
                mask = domain_mask[z0:z0 + n, y0:y0 + n, x0:x0 + n].contiguous()
                if int(mask.sum().item()) > n ** 3 // 20:
                    break
        else:
            mask = _random_crop_mask(n, rng, device)
        cs = [tuple(c) for c in rng.uniform(0.1, 0.9, size=(int(rng.integers(1, 6)), 3)) * (n + 1) * h]
        sigma = float(rng.uniform(3, 10)) * h
        b = torch.zeros((n, n, n), dtype=torch.float64, device=device)
        noise = inputs.random_field((n, n, n), seed=int(rng.integers(1 << 30)), device=device)
        if rng.random() < noise_fraction:
            b = noise
        else:
            for c in cs:
                amp = float(rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.5)) if signed else 1.0
                b = b + amp * inputs.gaussian_source(n, n, n, [c], sigma=sigma, h=h, device=device)
            b = b + 0.05 * noise
        b = b * mask.double()
        H = api.Handle(n, n, n, degree, h, dt, mask=mask, precision="f32_ir")
        xs = torch.zeros_like(b)
        H.cg_solve(b, xs, tol=1e-10)
        H.close()
        out.append(CropProblem(mask, b, xs))
    return out


def make_pairs(count: int, crop: int = 48, h: float = 1.0 / 513, dt: float = 1e-3, seed: int = 0,
               ks=(1, 2, 3, 4, 6, 8, 12, 16, 24, 32), degree: int = 3, device="cuda",
               signed: bool = True, noise_fraction: float = 0.0, problems=None) -> PairSet:
    """`count` pairs from the plain solver on random masked crop problems (make_problems), one
    pair per iteration count in ks (0: the right-hand side itself)."""
    n = crop
    if problems is None:
        problems = make_problems((count + len(ks) - 1) // len(ks), crop, h, dt, seed, degree, device,
                                 signed, noise_fraction)
    R = torch.empty((count, n, n, n), dtype=torch.float32, device=device)
    E = torch.empty_like(R)
    M = torch.empty((count, n, n, n), dtype=torch.uint8, device=device)
    vol = h ** 3
    i = 0
    for P in problems:
        if i >= count:
            break
        H32 = api.Handle(n, n, n, degree, h, dt, mask=P.mask, precision="f32")
        Hop = api.Handle(n, n, n, degree, h, dt, mask=P.mask, precision="f64")
        b32 = P.b.float()
        for k in ks:
            if i >= count:
                break
            xk = torch.zeros_like(b32)
            if k > 0:
                H32.cg_solve(b32, xk, tol=1e-30, max_iter=k)
            xk64 = xk.double()
            rk = P.b - Hop.op_apply(xk64)
            nr = torch.linalg.vector_norm(rk).item()
            if not (nr > 0) or not math.isfinite(nr):
                continue
            R[i] = (rk / nr).float()
            E[i] = ((P.xs - xk64) * (vol / nr)).float()
            M[i] = P.mask
            i += 1
        H32.close()
        Hop.close()
    return PairSet(R[:i], E[:i], M[:i], (n, n, n), h, dt, degree)


def fcg_pairs(net: api.Net, problems: list, steps: int = 30, h: float = 1.0 / 513, dt: float = 1e-3,
              degree: int = 3) -> PairSet:
    """On-policy pairs: the residuals that flexible CG(1) preconditioned by `net` itself meets on
    the given problems (the first `steps` iterations from x = 0), with their errors. A network
    trained only on the plain solver's residuals is good on those but poor on the residuals it
    leaves behind, which are exactly the ones flexible CG then hands it; adding these pairs and
    training again (a few rounds) removes that mismatch. The iteration is the library's own
    (fcg_record: the inner FP32 solve of fcg_solve, with its fallbacks); this function only turns
    each recorded state (r_k, d_k of A d = b / ||b||) into a pair (r_k / ||r_k||, the scaled
    error of x_k = ||b|| d_k)."""
    n = problems[0].mask.shape[0]
    vol = h ** 3
    Rs, Es, Ms = [], [], []
    for P in problems:
        H = api.Handle(n, n, n, degree, h, dt, mask=P.mask, precision="f32_ir")
        try:
            r, d, bnorm = H.fcg_record(P.b, steps, net)
        finally:
            H.close()
        for k in range(r.shape[0]):
            nr = torch.linalg.vector_norm(r[k]).item()
            if not (nr > 1e-7) or not math.isfinite(nr):
                break
            Rs.append((r[k] / nr).contiguous())
            Es.append(((P.xs - bnorm * d[k].double()) * (vol / (bnorm * nr))).float())
            Ms.append(P.mask)
    return PairSet(torch.stack(Rs), torch.stack(Es), torch.stack(Ms), (n, n, n), h, dt, degree)


def concat(a: PairSet, b: PairSet) -> PairSet:
    return PairSet(torch.cat([a.r, b.r]), torch.cat([a.e, b.e]), torch.cat([a.mask, b.mask]), a.shape,
                   a.h, a.dt, a.degree)


def train_on_policy(net: api.Net, pairs: PairSet, problems: list, rounds: int = 3, epochs: int = 4,
                    round_epochs: int = 3, batch: int = 16, lr: float = 2e-3, steps: int = 30,
                    log=None) -> list:
    """Energy-norm training on the plain solver's pairs, then `rounds` rounds of: collect the
    residuals of flexible CG with the current network on `problems` (fcg_pairs), add them, and
    train again at half the learning rate. Returns the per-epoch losses of all rounds."""
    losses = train(net, pairs, epochs=epochs, batch=batch, lr=lr, log=log)
    for rd in range(rounds):
        pairs = concat(pairs, fcg_pairs(net, problems, steps, pairs.h, pairs.dt, pairs.degree))
        losses += train(net, pairs, epochs=round_epochs, batch=batch, lr=lr / 2, seed=rd + 1, log=log)
    return losses


def init_params(seed: int = 0, out_scale: float = 0.1, h: float = 1.0 / 513, dt: float = 1e-3,
                degree: int = 3) -> torch.Tensor:
    """He-style weights, zero biases, small coarse output layer, and the full-resolution filter
    started at the Jacobi scale (1 / A_ii in the network's output unit); the layout of
    bsk_net_param_count."""
    g = torch.Generator().manual_seed(seed)
    C, KT = 16, 27
    parts = [torch.randn(KT * C, generator=g) * math.sqrt(2.0 / KT), torch.zeros(C)]
    for _ in range(3):
        parts += [torch.randn(KT * C * C, generator=g) * math.sqrt(2.0 / (KT * C)), torch.zeros(C)]
    parts += [torch.randn(KT * C, generator=g) * math.sqrt(1.0 / (KT * C)) * out_scale, torch.zeros(1)]
    # 1 / A_ii at a node n + 1 away from every face (the library's Jacobi diagonal), in the
    # network's output unit (the operator scaled by 1 / (hx hy hz))
    m = 2 * degree + 3
    H = api.Handle(m, m, m, degree, h, dt, precision="f64")
    try:
        H.set_preconditioner("jacobi")
        inv_aii = float(H.inverse_diagonal()[m // 2, m // 2, m // 2]) * h ** 3
    finally:
        H.close()
    wf = torch.zeros(KT)
    wf[13] = inv_aii
    parts.append(wf)
    return torch.cat(parts).float()


class EnergyLoss:
    """Relative energy-norm error of the network's output, the quantity that bounds what one
    flexible-CG step with direction z gains: with the scaled operator A' = A / (hx hy hz), for
    which A' e = r (input and target of a pair),

        L = (z - e)^T A' (z - e) / (e^T A' e),    dL/dz = 2 (A' z - r) / (e . r).

    L < 1 guarantees z . r > 0 (a descent direction); L = 0 is the exact error. The operator
    runs through an unmasked handle of the crop; masking its input and output gives the masked
    problem's operator (a principal submatrix)."""

    def __init__(self, pairs: PairSet):
        n = pairs.shape
        self.H = api.Handle(n[2], n[1], n[0], pairs.degree, pairs.h, pairs.dt, precision="f32")
        self.inv_vol = 1.0 / pairs.h ** 3

    def __call__(self, z, r, e, mask):
        m = mask.float()
        Az = self.H.op_apply(z * m) * (m * self.inv_vol)
        g = Az - r
        c = torch.dot(e.reshape(-1), r.reshape(-1)).item()
        L = torch.dot((z - e).reshape(-1), g.reshape(-1)).item() / c
        return L, g, 2.0 / c

    def close(self):
        self.H.close()


def train(net: api.Net, pairs: PairSet, epochs: int = 4, batch: int = 16, lr: float = 2e-3,
          seed: int = 0, log=None, loss: str = "energy") -> list:
    """Adam on mini-batches of `batch` pairs; per epoch the learning rate halves. loss="energy"
    minimises the mean relative energy-norm error (EnergyLoss), loss="mse" the mean squared
    error of N(r) against e. Returns the mean loss of each epoch."""
    rng = np.random.default_rng(seed)
    count = pairs.r.shape[0]
    losses = []
    t0 = time.time()
    energy = EnergyLoss(pairs) if loss == "energy" else None
    try:
        for ep in range(epochs):
            order = rng.permutation(count)
            ep_loss, nb = 0.0, 0
            lr_ep = lr * (0.5 ** ep)
            for s in range(0, count - batch + 1, batch):
                net.zero_grad()
                bl = 0.0
                for j in order[s:s + batch]:
                    j = int(j)
                    if energy is None:
                        net.backward(pairs.r[j], pairs.e[j], pairs.mask[j])
                    else:
                        z = net.forward(pairs.r[j], pairs.mask[j])
                        L, g, w = energy(z, pairs.r[j], pairs.e[j], pairs.mask[j])
                        net.backward_grad(pairs.r[j], g.contiguous(), pairs.mask[j], w)
                        bl += L
                if energy is None:
                    bl = net.read()
                net.adam(lr_ep, 1.0 / batch)
                ep_loss += bl / batch
                nb += 1
            losses.append(ep_loss / max(nb, 1))
            if log:
                log(f"epoch {ep}: loss {losses[-1]:.4e} ({time.time() - t0:.1f} s)")
    finally:
        if energy is not None:
            energy.close()
    return losses


def energy_error(net: api.Net, pairs: PairSet) -> float:
    """Mean relative energy-norm error of the network over a pair set (EnergyLoss)."""
    energy = EnergyLoss(pairs)
    try:
        tot = 0.0
        for j in range(pairs.r.shape[0]):
            z = net.forward(pairs.r[j], pairs.mask[j])
            tot += energy(z, pairs.r[j], pairs.e[j], pairs.mask[j])[0]
        return tot / max(pairs.r.shape[0], 1)
    finally:
        energy.close()
