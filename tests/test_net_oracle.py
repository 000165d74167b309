"""Pins of the network reference (oracle/net_ref.py): its backward pass against central finite
differences of its own loss (FP64, no BF16 rounding), and adjoint identities of the gather /
scatter convolution pair, on tiny grids. A planted mistake (dropped skip gradient) must fail."""
import numpy as np
import pytest

from oracle import net_ref as nr


def _problem(shape, seed):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(shape)
    e = rng.standard_normal(shape)
    mask = (rng.random(shape) < 0.8).astype(np.float64)
    r *= mask
    return r, e, mask


def test_adjoint_identities():
    rng = np.random.default_rng(1)
    for mode, din, dout in (("s1", (5, 4, 6), (5, 4, 6)), ("s2", (7, 6, 5), (4, 3, 3)),
                            ("t2", (4, 3, 3), (7, 6, 5))):
        x = rng.standard_normal(din + (3,))
        W = rng.standard_normal((27, 2, 3))
        g = rng.standard_normal(dout + (2,))
        lhs = np.sum(nr.conv(x, W, mode, dout) * g)
        rhs = np.sum(x * nr.conv_adjoint(g, W, mode, din))
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1)
        # the transposed stride-2 gather is the adjoint of the stride-2 gather
        if mode == "s2":
            W2 = np.transpose(W, (0, 2, 1))
            lhs2 = np.sum(nr.conv(x, W, "s2", dout) * g)
            rhs2 = np.sum(x * nr.conv(g, W2, "t2", din))
            assert abs(lhs2 - rhs2) <= 1e-11 * (abs(lhs2) + 1)


def test_backward_matches_finite_differences():
    shape = (6, 5, 7)
    r, e, mask = _problem(shape, 2)
    params = nr.init_params(3, out_scale=1.0)
    params += np.random.default_rng(4).standard_normal(params.size) * 0.05   # non-zero biases
    L, g, _ = nr.loss_and_grad(params, r, e, mask, emulate_bf16=False)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(params.size, 40, replace=False),
                          [0, 432, 448, nr.NPARAM - 1]])   # W1, b1, W2 start, b5
    eps = 1e-6
    for i in idx:
        p1 = params.copy(); p1[i] += eps
        p2 = params.copy(); p2[i] -= eps
        fd = (nr.loss_and_grad(p1, r, e, mask, False)[0] - nr.loss_and_grad(p2, r, e, mask, False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_planted_missing_skip_gradient_is_caught():
    shape = (6, 5, 7)
    r, e, mask = _problem(shape, 8)
    params = nr.init_params(9, out_scale=1.0)
    L, g, _ = nr.loss_and_grad(params, r, e, mask, emulate_bf16=False)
    # recompute the W1 gradient without the skip term and compare with finite differences
    z, c = nr.forward(params, r, mask, False)
    i = 5   # a W1 entry
    eps = 1e-6
    p1 = params.copy(); p1[i] += eps
    p2 = params.copy(); p2[i] -= eps
    fd = (nr.loss_and_grad(p1, r, e, mask, False)[0] - nr.loss_and_grad(p2, r, e, mask, False)[0]) / (2 * eps)
    assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8
    # planted: drop the skip contribution to da1 and redo the first-layer gradient
    W1, W2, W3, W4, W5 = c["W"]
    m = mask
    cnt = m.sum()
    dz = 2.0 * (z - e) * m / cnt
    da4 = nr.conv_adjoint(dz[..., None], W5[:, None, :], "t2", c["d"][1])
    g4 = da4 * (c["a4"] > 0)
    g3 = nr.conv_adjoint(g4, W4, "t2", c["d"][2]) * (c["a3"] > 0)
    g2 = nr.conv_adjoint(g3, W3, "s1", c["d"][2]) * (c["a2"] > 0)
    g1_bad = nr.conv_adjoint(g2, W2, "s2", c["d"][1]) * (c["a1"] > 0)   # + g4 dropped
    bad = nr.conv_wgrad(c["x0"], g1_bad, "s2")[:, :, 0].reshape(-1)[i]
    assert abs(bad - fd) > 1e-4 * max(1.0, abs(fd))


def test_bf16_rounding_reference():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-8])
    y = nr.bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0          # ties to even
    assert y[2] == 1.0078125
    assert abs(y[3] + 3.140625) < 1e-12
    assert np.all(np.abs(y - x) <= np.abs(x) * 2 ** -8)


def test_linear_network_is_a_linear_map():
    """act="linear": identity activations and no biases, so N(a r1 + b r2) = a N(r1) + b N(r2)
    and N(0) = 0 even with non-zero bias parameters."""
    shape = (7, 6, 5)
    rng = np.random.default_rng(11)
    params = nr.init_params(12, out_scale=1.0) + rng.standard_normal(nr.NPARAM) * 0.05
    r1, r2 = rng.standard_normal(shape), rng.standard_normal(shape)
    mask = (rng.random(shape) < 0.8).astype(np.float64)
    f = lambda r: nr.forward(params, r, mask, emulate_bf16=False, act="linear")[0]  # noqa: E731
    lhs = f(2.0 * r1 - 0.5 * r2)
    rhs = 2.0 * f(r1) - 0.5 * f(r2)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    assert np.max(np.abs(f(np.zeros(shape)))) == 0.0
    # the relu network with the same parameters is not linear
    g = lambda r: nr.forward(params, r, mask, emulate_bf16=False)[0]  # noqa: E731
    assert np.max(np.abs(g(2.0 * r1 - 0.5 * r2) - (2.0 * g(r1) - 0.5 * g(r2)))) > 1e-6


def test_linear_backward_matches_finite_differences():
    shape = (6, 5, 7)
    r, e, mask = _problem(shape, 13)
    params = nr.init_params(14, out_scale=1.0)
    params += np.random.default_rng(15).standard_normal(params.size) * 0.05
    L, g, _ = nr.loss_and_grad(params, r, e, mask, emulate_bf16=False, act="linear")
    off = 0
    for name, shp in nr.SIZES:
        size = int(np.prod(shp))
        if name.startswith("b"):
            assert np.all(g[off:off + size] == 0.0), name
        off += size
    rng = np.random.default_rng(16)
    eps = 1e-6
    for i in np.concatenate([rng.choice(params.size, 30, replace=False), [0, 450, nr.NPARAM - 14]]):
        p1 = params.copy(); p1[i] += eps
        p2 = params.copy(); p2[i] -= eps
        fd = (nr.loss_and_grad(p1, r, e, mask, False, "linear")[0]
              - nr.loss_and_grad(p2, r, e, mask, False, "linear")[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def _conv_f32(x, W, mode, dout):
    """The reference's gather convolution with FP32 accumulation: the kind of rounding the GPU's
    sums have, used to check that the element-wise comparison tolerates it."""
    out = np.zeros(tuple(dout) + (W.shape[1],), dtype=np.float32)
    x = x.astype(np.float32)
    W = W.astype(np.float32)
    for k, kz, ky, kx in nr._taps():
        iz, oz = nr._src(mode, dout[0], kz, x.shape[0])
        iy, oy = nr._src(mode, dout[1], ky, x.shape[1])
        ix, ox = nr._src(mode, dout[2], kx, x.shape[2])
        g = x[np.ix_(iz, iy, ix)] * (oz[:, None, None] & oy[None, :, None] & ox[None, None, :])[..., None]
        out += (g @ W[k].T).astype(np.float32)
    return out.astype(np.float64)


@pytest.mark.parametrize("act", ["relu", "linear"])
def test_elementwise_comparison_tolerates_fp32_sums_and_catches_a_wrong_tap(act, monkeypatch):
    """The GPU-vs-reference comparison of tests/netcheck.py passes the reference evaluated with
    FP32 sums, and fails when a 16->16 convolution reads one tap from the wrong weight block (a
    planted mistake in the reference: tap 13 of W2 replaced by tap 14), or when the weight
    gradient of one tap comes from the wrong tap."""
    import netcheck
    rng = np.random.default_rng(0)
    shape = (16, 16, 16)
    p = nr.init_params(3, out_scale=1.0) + rng.standard_normal(nr.NPARAM) * 0.02
    mask = (rng.random(shape) < 0.85).astype(np.float64)
    r = rng.standard_normal(shape) * mask * 0.05
    zr, _ = nr.forward(p, r, mask, act=act)
    S, _ = netcheck.abs_forward(p, r, mask, act)
    with monkeypatch.context() as m:
        m.setattr(nr, "conv", _conv_f32)
        z32, _ = nr.forward(p, r, mask, act=act)
    assert netcheck.forward_ok(z32, zr, S, mask)
    q = nr.unpack(p)
    q = {k: v.copy() for k, v in q.items()}
    q["W2"][13] = q["W2"][14]
    zp, _ = nr.forward(nr.pack(q), r, mask, act=act)
    assert not netcheck.forward_ok(zp, zr, S, mask)
    # gradients: one tap of dL/dW3 taken from the neighbouring tap
    e = rng.standard_normal(shape) * 0.05
    _, gr, _ = nr.loss_and_grad(p, r, e, mask, act=act)
    Gs = netcheck.abs_gradient_scale(p, r, e, mask, act)
    assert max(netcheck.gradient_errors(gr, gr, Gs).values()) == 0.0
    gp = nr.unpack(gr)
    gp = {k: v.copy() for k, v in gp.items()}
    gp["W3"][13] = gp["W3"][14]
    errs = netcheck.gradient_errors(nr.pack(gp), gr, Gs)
    assert not netcheck.gradient_ok(errs), errs
