"""Element-wise comparison of the GPU network with the FP64 reference (oracle/net_ref.py).

Both sides round the hidden-layer weights and the stored activations to bfloat16; they differ in
how the sums of products are accumulated (FP32 on the GPU, FP64 in the reference). Each output
is compared with the magnitude it is made of: S, the same network evaluated on |weights|, |r|
(and |biases|), so that every term enters with its absolute value. An FP32 accumulation of k
terms is off by at most about k 2^-24 S, and where that tips a stored activation across a
bfloat16 rounding boundary the output moves by one bfloat16 ulp of that activation times the
downstream absolute gain, which is again bounded by a small multiple of 2^-8 of the scale such
an activation contributes to S; measured over many grids both stay below 2e-6 S (median about
1e-12 S). A kernel that reads a wrong tap, or computes one with a wrong weight, changes every
output the tap feeds by about |w| |a| of that tap, which is well above that on most outputs.
Gradients are compared weight by weight the same way, with the absolute-value version of the
backward pass as the scale.
"""
import numpy as np

from oracle import net_ref as nr

# Tolerances relative to the absolute-value scale (see the module docstring).
FWD_MAX = 2.0 ** -16      # any single output
FWD_MEDIAN = 2.0 ** -24   # half of the outputs (rounding noise is ~1e-12 there)
# any single gradient: weights (each a sum over all voxels; measured <= 3e-6 of the scale on the
# GPU) and biases (sums of adjoints alone, where the bfloat16 adjoints weigh more; <= 1e-4)
GRAD_MAX = 2.0 ** -16
GRAD_MAX_BIAS = 2.0 ** -11


def abs_forward(params, r, mask, act):
    """S: the network on |params| and |r|; with every term non-negative ReLU is the identity,
    so S bounds the absolute sum behind each output (biases included in ReLU mode)."""
    S, cache = nr.forward(np.abs(params), np.abs(r), mask, emulate_bf16=False, act=act)
    return S, cache


def forward_errors(z, zr, S, mask):
    """|z - zr| / S over the active outputs (S = 0 only where both outputs are exactly zero)."""
    act = (mask > 0) & (S > 0)
    return np.abs(z - zr)[act] / S[act]


def forward_ok(z, zr, S, mask):
    e = forward_errors(z, zr, S, mask)
    return e.size == 0 or (e.max() <= FWD_MAX and np.median(e) <= FWD_MEDIAN)


def abs_gradient_scale(params, r, e, mask, act):
    """Per-weight scale of dL/dW: the backward pass of the reference with every factor taken by
    its absolute value (|dz|, |W|, activations of the absolute network, ReLU slopes as 1)."""
    z, _ = nr.forward(params, r, mask, act=act)
    m = np.ones_like(z) if mask is None else np.asarray(mask, dtype=np.float64)
    dz = 2.0 * np.abs(z - e) * m / m.sum()
    _, c = abs_forward(params, r, mask, act)
    W1, W2, W3, W4, W5 = (np.abs(w) for w in c["W"])
    d0, d1, d2 = c["d"]
    G = {}
    G["b5"] = np.array([dz.sum()])
    G["Wf"] = nr.conv_wgrad(c["x0"], dz[..., None], "s1")[:, 0, 0]
    G["W5"] = nr.conv_wgrad(c["a4"], dz[..., None], "t2")[:, 0, :]
    g4 = nr.conv_adjoint(dz[..., None], W5[:, None, :], "t2", d1)
    G["b4"] = g4.sum(axis=(0, 1, 2))
    G["W4"] = nr.conv_wgrad(c["a3"], g4, "t2")
    g3 = nr.conv_adjoint(g4, W4, "t2", d2)
    G["b3"] = g3.sum(axis=(0, 1, 2))
    G["W3"] = nr.conv_wgrad(c["a2"], g3, "s1")
    g2 = nr.conv_adjoint(g3, W3, "s1", d2)
    G["b2"] = g2.sum(axis=(0, 1, 2))
    G["W2"] = nr.conv_wgrad(c["a1"], g2, "s2")
    g1 = nr.conv_adjoint(g2, W2, "s2", d1) + g4
    G["b1"] = g1.sum(axis=(0, 1, 2))
    G["W1"] = nr.conv_wgrad(c["x0"], g1, "s2")[:, :, 0]
    if act == "linear":
        for k in ("b1", "b2", "b3", "b4", "b5"):
            G[k] = np.zeros_like(G[k])
    return nr.pack(G)


def gradient_ok(errs):
    return all(v <= (GRAD_MAX_BIAS if name.startswith("b") else GRAD_MAX) for name, v in errs.items())


def gradient_errors(g, gr, Gs):
    """Per parameter block: the largest |g - gr| / Gs over the weights with Gs > 0."""
    out, off = {}, 0
    for name, shp in nr.SIZES:
        n = int(np.prod(shp))
        a, b, s = g[off:off + n], gr[off:off + n], Gs[off:off + n]
        off += n
        keep = s > 0
        out[name] = float(np.max(np.abs(a - b)[keep] / s[keep])) if keep.any() else 0.0
    return out
