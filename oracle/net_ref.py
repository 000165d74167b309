"""FP64 NumPy reference of the learned preconditioner network (forward, loss, backward).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the test-suite uses it. The paper has no
learned component; this reference follows the network definition of the library's C ABI
(include/bsk.h, "the learned preconditioner"):

    a1 = relu(conv_s2(r; W1) + b1)          1 -> 16 channels
    a2 = relu(conv_s2(a1; W2) + b2)         16 -> 16
    a3 = relu(conv_s1(a2; W3) + b3)         16 -> 16
    a4 = relu(convT_s2(a3; W4) + b4 + a1)   16 -> 16 (transposed, plus skip)
    z  = mask * (convT_s2(a4; W5) + b5 + conv_s1(r; Wf))   16 -> 1, plus a full-resolution
                                                          1 -> 1 filter of r

with 3x3x3 taps, zero padding, conv_s2 reading input 2o + k - 1 for output o and tap k, conv_s1
reading o + k - 1, and convT_s2 the exact adjoint of conv_s2 (output o gathers input
(o + 1 - k) / 2 when that is an integer in range). Forward convolutions gather per tap; the
backward pass scatters per tap (the transpose of the gather, written out directly), so it shares
no formulation with the GPU kernels, which express the adjoints as transposed-weight
convolutions. Arrays are [z][y][x][channel]; weights [tap][out][in].
"""
from __future__ import annotations

import numpy as np

C = 16
KT = 27
SIZES = [("W1", (KT, C)), ("b1", (C,)), ("W2", (KT, C, C)), ("b2", (C,)), ("W3", (KT, C, C)),
         ("b3", (C,)), ("W4", (KT, C, C)), ("b4", (C,)), ("W5", (KT, C)), ("b5", (1,)),
         ("Wf", (KT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[off:off + n].reshape(shape)
        off += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(a):
    """Round to bfloat16 (round to nearest even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _src(mode, n_out, k, n_in):
    o = np.arange(n_out)
    if mode == "s1":
        i = o + k - 1
        ok = np.ones_like(o, dtype=bool)
    elif mode == "s2":
        i = 2 * o + k - 1
        ok = np.ones_like(o, dtype=bool)
    else:  # transposed stride 2
        t = o + 1 - k
        ok = (t % 2) == 0
        i = t // 2
    ok &= (i >= 0) & (i < n_in)
    return np.where(ok, i, 0), ok


def _taps():
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                yield (kz * 3 + ky) * 3 + kx, kz, ky, kx


def conv(x, W, mode, dout):
    """Gather form: out[o] = sum_k W[k] x[src(o, k)] (x: [z][y][x][cin], W: [27][cout][cin])."""
    nz, ny, nx = x.shape[:3]
    out = np.zeros(tuple(dout) + (W.shape[1],))
    for k, kz, ky, kx in _taps():
        iz, oz = _src(mode, dout[0], kz, nz)
        iy, oy = _src(mode, dout[1], ky, ny)
        ix, ox = _src(mode, dout[2], kx, nx)
        g = x[np.ix_(iz, iy, ix)] * (oz[:, None, None] & oy[None, :, None] & ox[None, None, :])[..., None]
        out += g @ W[k].T
    return out


def conv_adjoint(gout, W, mode, din):
    """Scatter form of the transpose: d x[src(o, k)] += W[k]^T g[o]; returns dx [din][cin]."""
    dx = np.zeros(tuple(din) + (W.shape[2],))
    dz_, dy_, dx_ = gout.shape[:3]
    for k, kz, ky, kx in _taps():
        iz, oz = _src(mode, dz_, kz, din[0])
        iy, oy = _src(mode, dy_, ky, din[1])
        ix, ox = _src(mode, dx_, kx, din[2])
        valid = (oz[:, None, None] & oy[None, :, None] & ox[None, None, :])
        contrib = (gout @ W[k]) * valid[..., None]
        np.add.at(dx, np.ix_(iz, iy, ix), contrib)
    return dx


def conv_wgrad(x, gout, mode):
    """dW[k] = sum_o g[o] x[src(o, k)]^T."""
    nz, ny, nx = x.shape[:3]
    dW = np.zeros((KT, gout.shape[3], x.shape[3]))
    for k, kz, ky, kx in _taps():
        iz, oz = _src(mode, gout.shape[0], kz, nz)
        iy, oy = _src(mode, gout.shape[1], ky, ny)
        ix, ox = _src(mode, gout.shape[2], kx, nx)
        g = x[np.ix_(iz, iy, ix)] * (oz[:, None, None] & oy[None, :, None] & ox[None, None, :])[..., None]
        dW[k] = np.einsum("zyxo,zyxi->oi", gout, g)
    return dW


def half(d):
    return tuple((v + 1) // 2 for v in d)


def forward(params, r, mask=None, emulate_bf16=True, act="relu"):
    """z and the cache of activations. With emulate_bf16 the weights of the hidden layers and the
    stored activations are rounded to bfloat16 as the GPU does. act="linear" replaces relu by the
    identity and drops the biases b1..b5 (the network is then a linear map of r)."""
    P = unpack(params)
    if act == "linear":
        P = {k: (np.zeros_like(v) if k.startswith("b") else v) for k, v in P.items()}
        relu = lambda a: a  # noqa: E731
    else:
        relu = lambda a: np.maximum(a, 0.0)  # noqa: E731
    rnd = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3, W4, W5 = (rnd(P[n]) for n in ("W1", "W2", "W3", "W4", "W5"))
    d0 = r.shape
    d1, d2 = half(d0), half(half(d0))
    x0 = np.asarray(r, dtype=np.float64)[..., None]
    a1 = rnd(relu(conv(x0, W1[:, :, None], "s2", d1) + P["b1"]))
    a2 = rnd(relu(conv(a1, W2, "s2", d2) + P["b2"]))
    a3 = rnd(relu(conv(a2, W3, "s1", d2) + P["b3"]))
    a4 = rnd(relu(conv(a3, W4, "t2", d1) + P["b4"] + a1))
    z = conv(a4, W5[:, None, :], "t2", d0)[..., 0] + P["b5"][0]
    z = z + conv(x0, P["Wf"][:, None, None], "s1", d0)[..., 0]
    if mask is not None:
        z = z * mask
    cache = dict(x0=x0, a1=a1, a2=a2, a3=a3, a4=a4, W=(W1, W2, W3, W4, W5), d=(d0, d1, d2), act=act)
    return z, cache


def loss_and_grad(params, r, e, mask=None, emulate_bf16=True, act="relu"):
    """L = mean over active voxels of (z - e)^2 and dL/dparams (FP64); with act="linear" the
    biases get no gradient."""
    z, c = forward(params, r, mask, emulate_bf16, act)
    m = np.ones_like(z) if mask is None else np.asarray(mask, dtype=np.float64)
    cnt = m.sum()
    d = (z - e) * m
    L = float((d * d).sum() / cnt)
    dz = 2.0 * d / cnt
    W1, W2, W3, W4, W5 = c["W"]
    d0, d1, d2 = c["d"]
    G = {}
    G["b5"] = np.array([dz.sum()])
    G["Wf"] = conv_wgrad(c["x0"], dz[..., None], "s1")[:, 0, 0]
    G["W5"] = conv_wgrad(c["a4"], dz[..., None], "t2")[:, 0, :]
    da4 = conv_adjoint(dz[..., None], W5[:, None, :], "t2", d1)
    on = (lambda a: np.ones_like(a)) if act == "linear" else (lambda a: (a > 0).astype(np.float64))
    g4 = da4 * on(c["a4"])
    G["b4"] = g4.sum(axis=(0, 1, 2))
    G["W4"] = conv_wgrad(c["a3"], g4, "t2")
    da3 = conv_adjoint(g4, W4, "t2", d2)
    g3 = da3 * on(c["a3"])
    G["b3"] = g3.sum(axis=(0, 1, 2))
    G["W3"] = conv_wgrad(c["a2"], g3, "s1")
    da2 = conv_adjoint(g3, W3, "s1", d2)
    g2 = da2 * on(c["a2"])
    G["b2"] = g2.sum(axis=(0, 1, 2))
    G["W2"] = conv_wgrad(c["a1"], g2, "s2")
    da1 = conv_adjoint(g2, W2, "s2", d1) + g4
    g1 = da1 * on(c["a1"])
    G["b1"] = g1.sum(axis=(0, 1, 2))
    G["W1"] = conv_wgrad(c["x0"], g1, "s2")[:, :, 0]
    if act == "linear":
        for k in ("b1", "b2", "b3", "b4", "b5"):
            G[k] = np.zeros_like(G[k])
    return L, pack(G), z


def init_params(seed: int = 0, out_scale: float = 0.1):
    """He-style initial weights, zero biases; the output layer scaled down."""
    rng = np.random.default_rng(seed)
    d = {}
    d["W1"] = rng.standard_normal((KT, C)) * np.sqrt(2.0 / KT)
    d["W2"] = rng.standard_normal((KT, C, C)) * np.sqrt(2.0 / (KT * C))
    d["W3"] = rng.standard_normal((KT, C, C)) * np.sqrt(2.0 / (KT * C))
    d["W4"] = rng.standard_normal((KT, C, C)) * np.sqrt(2.0 / (KT * C))
    d["W5"] = rng.standard_normal((KT, C)) * np.sqrt(1.0 / (KT * C)) * out_scale
    for b in ("b1", "b2", "b3", "b4"):
        d[b] = np.zeros(C)
    d["b5"] = np.zeros(1)
    d["Wf"] = np.zeros(KT)
    return pack(d)
