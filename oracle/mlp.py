"""CPU reference of the density-proposal network (test infrastructure only).

Not in the paper: the network only proposes rho', a lower bound of the
optimal h-clique density (Problem 1); the seeded decomposition checks the
proposal exactly, so no answer depends on it.  This module restates, in
float64 numpy, what the library's network computes, so that its forward
pass, gradients and Adam step can be compared element by element.

Network: x (64) -> h1 = relu(x W1 + b1) (256) -> h2 = relu(h1 W2 + b2) (256)
-> h3 = relu(h2 W3 + b3) (256) -> out = h3 W4 + b4 (1).  The parameters are
one flat float32 vector in that order (W stored input-major, [in x out]).
The forward pass reads the weight matrices rounded to bfloat16 (round to
nearest, ties to even) and the biases in float32; gradients are taken with
respect to those values and applied to the float32 master copy.

Loss: pinball (quantile) loss at quantile q, mean over the batch,
rho_q(u) = u (q - [u < 0]) with u = y - out.

Only ``tests/`` may import this module.
"""
from __future__ import annotations

import numpy as np

NFEAT = 64
NHID = 256
SHAPES = [("W1", (NFEAT, NHID)), ("b1", (NHID,)), ("W2", (NHID, NHID)), ("b2", (NHID,)),
          ("W3", (NHID, NHID)), ("b3", (NHID,)), ("W4", (NHID, 1)), ("b4", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(p):
    """Views of the flat parameter vector, by name."""
    out, at = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = p[at:at + size].reshape(shape)
        at += size
    return out


def bf16_round(a):
    """float32 -> nearest bfloat16 value (ties to even), returned as float32.
    NaN and infinities are not expected here."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def effective(p):
    """The values the forward pass uses: bf16 weights, float32 biases, as float64."""
    P = unflatten(np.asarray(p, np.float32))
    return {k: (bf16_round(v) if k.startswith("W") else v).astype(np.float64)
            for k, v in P.items()}


def forward(p, X):
    """Returns (out [B], cache) for feature rows X [B x 64]."""
    E = effective(p)
    X = np.asarray(X, np.float64)
    z1 = X @ E["W1"] + E["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ E["W2"] + E["b2"]
    h2 = np.maximum(z2, 0)
    z3 = h2 @ E["W3"] + E["b3"]
    h3 = np.maximum(z3, 0)
    out = (h3 @ E["W4"] + E["b4"])[:, 0]
    return out, dict(E=E, X=X, h1=h1, h2=h2, h3=h3)


def pinball(out, y, q):
    """Mean pinball loss and its derivative with respect to out."""
    y = np.asarray(y, np.float64)
    u = y - out
    ind = (u < 0).astype(np.float64)
    loss = float(np.mean(u * (q - ind)))
    dout = -(q - ind) / len(y)
    return loss, dout


def loss_and_grad(p, X, y, q):
    """Loss and the flat gradient (float64) by backpropagation."""
    out, c = forward(p, X)
    loss, dout = pinball(out, y, q)
    E = c["E"]
    g = {}
    d = dout[:, None]                                  # [B x 1]
    g["W4"] = c["h3"].T @ d
    g["b4"] = d.sum(0)
    d3 = (d @ E["W4"].T) * (c["h3"] > 0)
    g["W3"] = c["h2"].T @ d3
    g["b3"] = d3.sum(0)
    d2 = (d3 @ E["W3"].T) * (c["h2"] > 0)
    g["W2"] = c["h1"].T @ d2
    g["b2"] = d2.sum(0)
    d1 = (d2 @ E["W2"].T) * (c["h1"] > 0)
    g["W1"] = c["X"].T @ d1
    g["b1"] = d1.sum(0)
    flat = np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])
    return loss, flat


def adam(p, m, v, step, grad, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) of step number `step` (1-based).
    Returns (p, m, v) in float64."""
    p = np.asarray(p, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
