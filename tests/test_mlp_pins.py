"""Pins of the float64 network reference (oracle/mlp.py) against things it
does not compute itself: finite differences of the forward pass, the
quantile property of the pinball loss, the closed-form first Adam step, the
bfloat16 format, and a hand-built network with a known output."""
from __future__ import annotations

import numpy as np

from oracle import mlp


def _params(seed, scale=0.1):
    r = np.random.default_rng(seed)
    return (r.standard_normal(mlp.NPARAMS) * scale).astype(np.float32)


def test_param_count():
    assert mlp.NPARAMS == 64 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1 == 148481


def test_bf16_round_exact_cases():
    vals = np.array([1.0, -2.5, 0.0, 3.0e38, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8,
                     1.0 + 2.0 ** -9], np.float32)
    got = mlp.bf16_round(vals)
    # 8 significand bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1);
    # 1 + 3*2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6 -> even (1 + 2^-6)
    want = np.array([1.0, -2.5, 0.0, np.float32(3.0e38), 1.0, 1.0 + 2.0 ** -6, 1.0], np.float32)
    assert np.array_equal(got[[0, 1, 2, 4, 5, 6]], want[[0, 1, 2, 4, 5, 6]])
    # the result has at most 8 significant bits
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    b = mlp.bf16_round(x).view(np.uint32)
    assert np.all(b & 0xFFFF == 0)
    assert np.all(np.abs(mlp.bf16_round(x) - x) <= np.abs(x) * 2.0 ** -8)


def test_hand_built_network():
    # W1 picks x0 into unit 0, W2/W3 pass unit 0 on, W4 doubles it, b4 = 1:
    # out = 2 relu(x0) + 1
    p = np.zeros(mlp.NPARAMS, np.float32)
    P = mlp.unflatten(p)
    P["W1"][0, 0] = 1.0
    P["W2"][0, 0] = 1.0
    P["W3"][0, 0] = 1.0
    P["W4"][0, 0] = 2.0
    P["b4"][0] = 1.0
    X = np.zeros((3, 64))
    X[:, 0] = [-1.0, 0.5, 3.0]
    out, _ = mlp.forward(p, X)
    assert np.allclose(out, [1.0, 2.0, 7.0])


def test_gradient_matches_finite_differences():
    # the forward pass reads bf16 weights; differentiate with respect to the
    # values it reads by perturbing biases (float32, exact) and checking weight
    # gradients through a network whose weights are already bf16 values with
    # a perturbation of one bf16 step
    r = np.random.default_rng(3)
    p = mlp.bf16_round(_params(1))
    X = r.standard_normal((12, 64))
    y = r.standard_normal(12) * 3
    q = 0.3
    loss, g = mlp.loss_and_grad(p, X, y, q)
    # the pinball loss is piecewise linear; keep perturbations small enough
    # that no residual changes sign, and compare central differences
    out, _ = mlp.forward(p, X)
    assert np.min(np.abs(y - out)) > 1e-3
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    picks = []
    for (name, _), a, b in zip(mlp.SHAPES, offs[:-1], offs[1:]):
        idx = r.choice(np.arange(a, b), size=min(6, b - a), replace=False)
        picks += [(name, int(i)) for i in idx]
    checked = 0
    for name, i in picks:
        base = float(p[i])
        if name.startswith("W"):
            # one bf16 ulp: base +- e are bf16 values too, so the forward pass
            # reads exactly the perturbed value
            e = 2.0 ** (np.floor(np.log2(max(abs(base), 2.0 ** -20))) - 7)
        else:
            e = 2.0 ** -12
        hi = p.copy()
        lo = p.copy()
        hi[i] = base + e
        lo[i] = base - e
        assert mlp.bf16_round(hi[i:i + 1])[0] == hi[i] or not name.startswith("W")
        lh, _ = mlp.loss_and_grad(hi, X, y, q)
        ll, _ = mlp.loss_and_grad(lo, X, y, q)
        fd = (lh - ll) / (float(hi[i]) - float(lo[i]))
        # the loss is piecewise linear in one parameter: central differences
        # are exact unless a ReLU kink falls inside the interval (rare)
        if np.isclose(fd, g[i], rtol=1e-6, atol=1e-9):
            checked += 1
    assert checked >= len(picks) - 2


def test_pinball_minimiser_is_quantile():
    # the constant prediction minimising the mean pinball loss is a q-quantile
    r = np.random.default_rng(5)
    y = r.standard_normal(999)
    for q in (0.05, 0.5, 0.9):
        grid = np.linspace(-4, 4, 8001)
        losses = [mlp.pinball(np.full(y.size, c), y, q)[0] for c in grid]
        c = grid[int(np.argmin(losses))]
        lo, hi = np.quantile(y, q, method="lower"), np.quantile(y, q, method="higher")
        assert lo - 1e-3 <= c <= hi + 1e-3


def test_pinball_derivative_sign():
    out = np.array([0.0, 0.0])
    y = np.array([1.0, -1.0])
    loss, d = mlp.pinball(out, y, 0.05)
    assert np.isclose(loss, (1.0 * 0.05 + 1.0 * 0.95) / 2)
    assert np.allclose(d, [-0.05 / 2, 0.95 / 2])


def test_first_adam_step_is_signed_lr():
    # after one step m_hat = g and v_hat = g^2, so each parameter moves by
    # lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps
    r = np.random.default_rng(7)
    g = r.standard_normal(50) + np.sign(r.standard_normal(50)) * 0.5
    p0 = r.standard_normal(50)
    p1, m, v = mlp.adam(p0, np.zeros(50), np.zeros(50), 1, g, lr=1e-3)
    assert np.allclose(p0 - p1, 1e-3 * np.sign(g), rtol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
