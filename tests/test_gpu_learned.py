"""The learned preconditioner: network forward and gradients vs the FP64 NumPy reference, GPU
training, flexible CG with and without the network, fallback, and what the trained network
gains over the method without it."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import net_ref as nr  # noqa: E402

import netcheck  # noqa: E402


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03057_gb300 import api, inputs, learned
    return api, inputs, learned


def _sample(shape, seed, inputs):
    rng = np.random.default_rng(seed)
    mask = (rng.random(shape) < 0.85).astype(np.uint8)
    r = rng.standard_normal(shape).astype(np.float32) * mask * 0.05
    e = rng.standard_normal(shape).astype(np.float32) * 0.05
    return r, e, mask


def _params(seed):
    p = nr.init_params(seed, out_scale=1.0)
    p += np.random.default_rng(seed + 1).standard_normal(p.size) * 0.02
    return p


@pytest.mark.parametrize("shape,act", [((9, 10, 13), "relu"), ((16, 16, 16), "relu"), ((7, 12, 20), "relu"),
                                       ((9, 10, 13), "linear"), ((16, 16, 16), "linear")])
def test_forward_matches_reference(mods, shape, act):
    api, inputs, learned = mods
    params = _params(3)
    r, e, mask = _sample(shape, 4, inputs)
    net = api.Net(shape[2], shape[1], shape[0], activation=act)
    net.set_params(torch.from_numpy(params).float())
    z = net.forward(torch.from_numpy(r).cuda(), torch.from_numpy(mask).cuda()).cpu().numpy()
    pr = params.astype(np.float32).astype(np.float64)
    zr, _ = nr.forward(pr, r.astype(np.float64), mask, act=act)
    S, _ = netcheck.abs_forward(pr, r.astype(np.float64), mask, act)
    e = netcheck.forward_errors(z.astype(np.float64), zr, S, mask)
    print(shape, act, "max", e.max(), "median", np.median(e))
    assert netcheck.forward_ok(z.astype(np.float64), zr, S, mask), (e.max(), np.median(e))
    assert np.all(z[mask == 0] == 0)


@pytest.mark.parametrize("act", ["relu", "linear"])
def test_gradients_match_reference(mods, act):
    api, inputs, learned = mods
    shape = (10, 12, 14)
    params = _params(5)
    r, e, mask = _sample(shape, 6, inputs)
    net = api.Net(shape[2], shape[1], shape[0], activation=act)
    net.set_params(torch.from_numpy(params).float())
    net.zero_grad()
    net.backward(torch.from_numpy(r).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(mask).cuda())
    loss, g = net.read(grads=True)
    pr = params.astype(np.float32).astype(np.float64)
    L, gr, _ = nr.loss_and_grad(pr, r.astype(np.float64), e.astype(np.float64), mask.astype(np.float64),
                                act=act)
    assert abs(loss - L) <= 1e-4 * abs(L)
    Gs = netcheck.abs_gradient_scale(pr, r.astype(np.float64), e.astype(np.float64), mask.astype(np.float64), act)
    errs = netcheck.gradient_errors(g.astype(np.float64), gr, Gs)
    print(act, errs)
    assert netcheck.gradient_ok(errs), errs


def test_output_gradient_backward_matches_reference(mods):
    """bsk_net_backward_grad with dL/dz supplied gives the reference's parameter gradients."""
    api, inputs, learned = mods
    shape = (10, 12, 14)
    params = _params(7)
    r, e, mask = _sample(shape, 8, inputs)
    pr = params.astype(np.float32).astype(np.float64)
    L, gr, zr = nr.loss_and_grad(pr, r.astype(np.float64), e.astype(np.float64), mask.astype(np.float64))
    dz = (2.0 * (zr - e) * mask / mask.sum()).astype(np.float32)
    net = api.Net(shape[2], shape[1], shape[0])
    net.set_params(torch.from_numpy(params).float())
    net.zero_grad()
    net.backward_grad(torch.from_numpy(r).cuda(), torch.from_numpy(dz).cuda(), torch.from_numpy(mask).cuda())
    loss, g = net.read(grads=True)
    assert loss == 0.0
    Gs = netcheck.abs_gradient_scale(pr, r.astype(np.float64), e.astype(np.float64), mask.astype(np.float64),
                                     "relu")
    errs = netcheck.gradient_errors(g.astype(np.float64), gr, Gs)
    print(errs)
    assert netcheck.gradient_ok(errs), errs


def test_training_reduces_loss(mods):
    api, inputs, learned = mods
    pairs = learned.make_pairs(60, crop=24, seed=1, ks=(1, 2, 4, 8, 16))
    net = api.Net(24, 24, 24)
    net.set_params(learned.init_params(0))
    losses = learned.train(net, pairs, epochs=3, batch=8, lr=2e-3)
    assert all(math.isfinite(v) for v in losses)
    assert losses[-1] < 0.8 * losses[0], losses


def _oracle_rel_residual(n, h, dt, mask, b, x):
    """The oracle's FP64 true relative residual ||b - A x|| / ||b|| of a returned solution (the
    masked operator, principal submatrix of the box operator)."""
    import oracle
    p = oracle.Problem(n, n, n, 3, h, dt=dt, mask=mask.cpu().numpy())
    bn = b.cpu().numpy()
    r = (bn - oracle.op_separable(p, x.cpu().numpy())) * p.mask
    return float(np.linalg.norm(r) / np.linalg.norm(bn * p.mask))


def _masked_problem(inputs, n, seed, h):
    rng = np.random.default_rng(seed)
    k = 5
    centers = [tuple(rng.uniform(0.25, 0.75, size=3)) for _ in range(k)]
    radii = list(rng.uniform(0.15, 0.35, size=k))
    mask = inputs.union_of_spheres_mask(n, n, n, centers, radii, h=1.0 / (n + 1), device="cuda")
    cs = [tuple(c) for c in rng.uniform(0.3, 0.7, size=(4, 3)) * (n + 1) * h]
    b = inputs.gaussian_source(n, n, n, cs, sigma=5 * h, h=h, device="cuda") * mask.double()
    return mask, b


def test_fcg_without_network_is_cg(mods):
    api, inputs, learned = mods
    n, h, dt, tol = 40, 1.0 / 513, 1e-3, 1e-8
    mask, b = _masked_problem(inputs, n, 11, h)
    H = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir")
    x1 = torch.zeros_like(b)
    r1 = H.cg_solve(b, x1, tol=tol)
    x2 = torch.zeros_like(b)
    r2 = H.fcg_solve(b, x2, None, tol=tol)
    assert r1["status"] == 0 and r2["status"] == 0 and r2["rel_residual"] <= tol
    assert abs(r2["iterations"] - r1["iterations"]) <= 0.25 * r1["iterations"] + 3
    d = (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x1)).item()
    assert d <= 1e-5


def test_identity_network_reproduces_cg(mods):
    """A linear network that is the identity (only the full-resolution filter's centre tap, 1)
    gives z = c r, for which flexible CG is plain CG: same iteration count and solution."""
    api, inputs, learned = mods
    n, h, dt, tol = 40, 1.0 / 513, 1e-3, 1e-8
    mask, b = _masked_problem(inputs, n, 11, h)
    H = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir")
    net = api.Net(n, n, n, activation="linear")
    p = torch.zeros(nr.NPARAM)
    p[-27 + 13] = 1.0
    net.set_params(p)
    x1 = torch.zeros_like(b)
    r1 = H.fcg_solve(b, x1, None, tol=tol)
    x2 = torch.zeros_like(b)
    r2 = H.fcg_solve(b, x2, net, tol=tol)
    assert r1["status"] == 0 and r2["status"] == 0 and r2["fallback_iter"] == -1
    assert _oracle_rel_residual(n, h, dt, mask, b, x2) <= 1.5 * tol
    assert abs(r2["iterations"] - r1["iterations"]) <= 2, (r1, r2)
    d = (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x1)).item()
    assert d <= 1e-6


def test_bad_network_falls_back_and_converges(mods):
    api, inputs, learned = mods
    n, h, dt, tol = 32, 1.0 / 513, 1e-3, 1e-8
    mask, b = _masked_problem(inputs, n, 12, h)
    H = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir")
    net = api.Net(n, n, n)
    p = learned.init_params(3)
    p[-28 - 16 * 27:-28] *= -50.0          # an output layer that points the wrong way
    p[-27:] *= -1.0
    net.set_params(p)
    x = torch.zeros_like(b)
    rep = H.fcg_solve(b, x, net, tol=tol)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol
    assert _oracle_rel_residual(n, h, dt, mask, b, x) <= 1.5 * tol
    pn = torch.full_like(p, float("nan"))
    net.set_params(pn)
    x = torch.zeros_like(b)
    rep = H.fcg_solve(b, x, net, tol=tol)
    assert rep["status"] == 0 and rep["rel_residual"] <= tol and rep["fallback_iter"] >= 0
    assert _oracle_rel_residual(n, h, dt, mask, b, x) <= 1.5 * tol


def test_trained_network_reduces_iterations(mods):
    """What the trained network gains: on a masked 64^3 problem (h = 1/513, dt = 1e-3, the
    resolution and time step of the 512^3 union-of-spheres workload), flexible CG preconditioned
    by the trained linear network reaches a 1e-8 true residual (FP64 refinement) in markedly fewer
    iterations than the same iteration without it. Training: 32^3 crops, energy-norm loss, then
    three rounds on the residuals that flexible CG with the network itself produces."""
    api, inputs, learned = mods
    h, dt, tol = 1.0 / 513, 1e-3, 1e-8
    problems = learned.make_problems(40, crop=32, h=h, dt=dt, seed=2, noise_fraction=0.25)
    pairs = learned.make_pairs(440, crop=32, h=h, dt=dt, problems=problems,
                               ks=(0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32))
    tr = api.Net(32, 32, 32, activation="linear")
    tr.set_params(learned.init_params(0, h=h, dt=dt))
    losses = learned.train_on_policy(tr, pairs, problems[:12], rounds=3)
    print("training losses:", [round(v, 4) for v in losses])
    assert losses[-1] < 0.5 * losses[0]
    params = tr.get_params()
    n = 64
    mask, b = _masked_problem(inputs, n, 21, h)
    H = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir")
    net = api.Net(n, n, n, activation="linear")
    net.set_params(params)
    x0 = torch.zeros_like(b)
    plain = H.fcg_solve(b, x0, None, tol=tol)
    x1 = torch.zeros_like(b)
    learned_rep = H.fcg_solve(b, x1, net, tol=tol)
    print("plain:", plain, "learned:", learned_rep)
    assert plain["status"] == 0 and learned_rep["status"] == 0
    assert learned_rep["rel_residual"] <= tol
    assert _oracle_rel_residual(n, h, dt, mask, b, x1) <= 1.5 * tol
    assert _oracle_rel_residual(n, h, dt, mask, b, x0) <= 1.5 * tol
    assert learned_rep["fallback_iter"] == -1
    assert learned_rep["iterations"] < 0.75 * plain["iterations"], (plain, learned_rep)
    d = (torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)).item()
    assert d <= 1e-6


def test_race_512_learned_solution_judged_by_oracle(mods, orc):
    """The 512^3 union-of-spheres race (one implicit Euler step, 32 Gaussian sources, tol 1e-8):
    the flexible-CG solution with the trained network is judged by the oracle at 2000 sampled
    active nodes -- the library's FP64 true residual b - A x must equal the oracle's there (to
    1e-12 of the operator's scale), and its norm must meet the tolerance."""
    api, inputs, learned = mods
    N, dt, tol = 512, 1e-3, 1e-8
    h = 1.0 / (N + 1)
    problems = learned.make_problems(40, crop=32, h=h, dt=dt, seed=2, noise_fraction=0.25)
    pairs = learned.make_pairs(440, crop=32, h=h, dt=dt, problems=problems,
                               ks=(0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32))
    tr = api.Net(32, 32, 32, activation="linear")
    tr.set_params(learned.init_params(0, h=h, dt=dt))
    learned.train_on_policy(tr, pairs, problems[:12], rounds=3)
    params = tr.get_params()
    tr.close()
    del pairs, problems
    centers, radii = inputs.random_spheres(5, 40, 0.05, 0.2)
    mask = inputs.union_of_spheres_mask(N, N, N, centers, radii, h=h, device="cuda")
    q = inputs.gaussian_source(N, N, N, inputs.gaussian_centers(5, 32), sigma=0.03, h=h, mask=mask,
                               device="cuda")
    H64 = api.Handle(N, N, N, 3, h, dt, mask=mask, precision="f64")
    b = H64.mass_apply(q) * dt
    del q
    H64.close()
    H32 = api.Handle(N, N, N, 3, h, dt, mask=mask, precision="f32_ir")
    net = api.Net(N, N, N, activation="linear")
    net.set_params(params)
    x = torch.zeros_like(b)
    rep = H32.fcg_solve(b, x, net, tol=tol)
    assert rep["status"] == 0, rep
    r, rr, bb = H32.residual(b, x, fp64=True)
    assert math.sqrt(rr / bb) <= tol
    m = mask.cpu().numpy()
    active = np.flatnonzero(m.reshape(-1))
    pts = np.random.default_rng(0).choice(active, size=2000, replace=False)
    p = orc.Problem(N, N, N, 3, h, dt=dt, mask=m)
    xh = x.cpu().numpy()
    ref = b.reshape(-1)[torch.from_numpy(pts).cuda()].cpu().numpy() - orc.op_points(p, xh, pts)
    got = r.reshape(-1)[torch.from_numpy(pts).cuda()].cpu().numpy()
    M, K = orc.bspline_kernels(3, h)
    absW = np.sum(np.abs(M)) ** 3 + dt * 3 * np.sum(np.abs(K)) * np.sum(np.abs(M)) ** 2
    scale = absW * np.max(np.abs(xh)) + b.abs().max().item()
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale
    net.close()
    H32.close()


def test_fcg_record_states_match_the_oracle(mods):
    """fcg_record (the states the on-policy training pairs are made of): with no network the
    recorded iterates are plain CG's, so ||b|| d_k equals the oracle's CG iterate x_k, and every
    recorded residual is b / ||b|| - A d_k of the oracle's operator (FP32 states: 1e-5 of the
    scale)."""
    import oracle
    api, inputs, learned = mods
    n, h, dt, steps = 24, 1.0 / 25, 1e-3, 12
    mask, b = _masked_problem(inputs, n, 5, h)
    H = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir")
    r, d, bnorm = H.fcg_record(b, steps)
    H.close()
    assert r.shape[0] == steps
    p = oracle.Problem(n, n, n, 3, h, dt=dt, mask=mask.cpu().numpy())
    bn = b.cpu().numpy() * p.mask
    assert abs(bnorm - np.linalg.norm(bn)) <= 1e-12 * np.linalg.norm(bn)
    for k in range(steps):
        dk = d[k].double().cpu().numpy()
        rk = r[k].double().cpu().numpy()
        want_r = (bn / bnorm - oracle.op_separable(p, dk)) * p.mask
        assert np.abs(rk - want_r).max() <= 1e-5 * np.abs(bn / bnorm).max(), k
        xk, it, _, _ = oracle.cg(p, bn, tol=0.0, max_iter=k) if k > 0 else (np.zeros_like(bn), 0, 0, 0)
        assert np.abs(bnorm * dk - xk).max() <= 1e-4 * max(np.abs(xk).max(), 1e-300) + 1e-30, k
    # with a network the first state is the scaled right-hand side, and the states are finite
    net = api.Net(n, n, n)
    net.set_params(learned.init_params(0, h=h, dt=dt))
    r2, d2, _ = api.Handle(n, n, n, 3, h, dt, mask=mask, precision="f32_ir").fcg_record(b, steps, net)
    assert torch.allclose(r2[0].double(), torch.from_numpy(bn / bnorm).to(r2.device), atol=1e-6)
    assert torch.isfinite(r2).all() and torch.isfinite(d2).all() and torch.count_nonzero(d2[0]) == 0
