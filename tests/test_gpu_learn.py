"""GPU tests of the density-proposal network and the seeded decomposition.

* forward pass, gradients and the Adam step of the CUDA network against the
  float64 reference (oracle/mlp.py) on the same parameters and inputs;
* the graph statistics: deterministic, and the exactly known entries equal
  to their definitions;
* the seeded CoreApp call: its outputs equal the oracle's CoreApp outputs
  whatever the proposal is (accepted, rejected, absent or absurd), and the
  accept decision equals the exact test recomputed from the oracle's levels.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlp
from paper_1906_00341_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_00341_gb300 import build as b
    b.build()
    from paper_1906_00341_gb300 import _lib
    _lib.load()
    return _lib


def _rand_state(seed, scale=0.08):
    r = np.random.default_rng(seed)
    p = (r.standard_normal(mlp.NPARAMS) * scale).astype(np.float32)
    st = np.zeros(3 * mlp.NPARAMS + 1, np.float32)
    st[: mlp.NPARAMS] = p
    return st


def test_param_count_and_init(L):
    M = L.Model(seed=11)
    assert M.count == mlp.NPARAMS
    st = M.state()
    P = mlp.unflatten(st[: mlp.NPARAMS])
    # He-uniform bounds, zero biases, zero moments, step 0
    assert np.all(np.abs(P["W1"]) <= math.sqrt(6 / 64) + 1e-6)
    assert np.all(np.abs(P["W2"]) <= math.sqrt(6 / 256) + 1e-6)
    for b in ("b1", "b2", "b3", "b4"):
        assert np.all(P[b] == 0)
    assert np.all(st[mlp.NPARAMS:] == 0)
    assert abs(np.std(P["W2"]) - math.sqrt(6 / 256) / math.sqrt(3)) < 0.01
    # deterministic in the seed
    M2 = L.Model(seed=11)
    assert np.array_equal(M2.state(), st)
    M3 = L.Model(seed=12)
    assert not np.array_equal(M3.state(), st)


@pytest.mark.parametrize("B", [1, 31, 33, 256, 1024])
def test_forward_matches_reference(L, B):
    M = L.Model(seed=1)
    st = _rand_state(B)
    M.set_state(st)
    X = np.random.default_rng(100 + B).standard_normal((B, 64)).astype(np.float32)
    got = M.forward(X)
    want, _ = mlp.forward(st[: mlp.NPARAMS], X)
    scale = 1 + np.abs(want)
    assert np.max(np.abs(got - want) / scale) < 2e-5


def test_state_roundtrip(L):
    M = L.Model(seed=2)
    st = _rand_state(5)
    st[mlp.NPARAMS: 2 * mlp.NPARAMS] = 0.25
    st[2 * mlp.NPARAMS: 3 * mlp.NPARAMS] = 0.5
    st[-1] = 17
    M.set_state(st)
    assert np.array_equal(M.state(), st)
    with pytest.raises(ValueError):
        M.set_state(st[:-1])


@pytest.mark.parametrize("B,q", [(7, 0.05), (64, 0.5), (300, 0.9)])
def test_gradient_matches_reference(L, B, q):
    M = L.Model(seed=3)
    st = _rand_state(50 + B)
    M.set_state(st)
    r = np.random.default_rng(B)
    X = r.standard_normal((B, 64)).astype(np.float32)
    out, _ = mlp.forward(st[: mlp.NPARAMS], X)
    # labels well away from the predictions: the sign of every residual is
    # the same in float32 and float64
    y = (out + np.where(r.random(B) < 0.5, -1, 1) * (0.5 + r.random(B))).astype(np.float32)
    loss, grad = M.gradient(X, y, q)
    wl, wg = mlp.loss_and_grad(st[: mlp.NPARAMS], X, y, q)
    assert abs(loss - wl) <= 1e-5 * (1 + abs(wl))
    err = np.abs(grad - wg)
    assert np.max(err) <= 1e-4 * np.max(np.abs(wg)) + 1e-7
    # a plain gradient call changes nothing
    assert np.array_equal(M.state(), st)


def test_adam_step_matches_reference(L):
    M = L.Model(seed=4)
    st = _rand_state(77)
    M.set_state(st)
    r = np.random.default_rng(9)
    X = r.standard_normal((128, 64)).astype(np.float32)
    y = r.standard_normal(128).astype(np.float32) * 4
    lr, q = 3e-3, 0.05
    s = st.copy()
    for step in range(1, 4):
        _, g = M.gradient(X, y, q)
        M.train_step(X, y, q, lr)
        got = M.state()
        p, m, v = mlp.adam(s[: mlp.NPARAMS], s[mlp.NPARAMS: 2 * mlp.NPARAMS],
                           s[2 * mlp.NPARAMS: 3 * mlp.NPARAMS], step, g.astype(np.float64), lr)
        n = mlp.NPARAMS
        assert np.allclose(got[:n], p, rtol=1e-5, atol=1e-7)
        assert np.allclose(got[n: 2 * n], m, rtol=1e-5, atol=1e-9)
        # 1 - 0.999f differs from 0.001 by 4.7e-5 relative: the second moment
        # carries that constant's float32 rounding
        assert np.allclose(got[2 * n: 3 * n], v, rtol=1e-4, atol=1e-12)
        assert got[-1] == step
        s = got


def test_training_fits_a_quantile(L):
    # y = 2 x0 + noise: after training, about q of the labels lie below the
    # predictions
    M = L.Model(seed=5)
    r = np.random.default_rng(6)
    X = r.standard_normal((4096, 64)).astype(np.float32)
    y = (2 * X[:, 0] + r.standard_normal(4096)).astype(np.float32)
    q = 0.2
    first = None
    for it in range(400):
        i = r.integers(0, 4096, 256)
        loss = M.train_step(X[i], y[i], q, 1e-3)
        first = loss if first is None else first
    assert loss < 0.6 * first
    pred = np.concatenate([M.forward(X[a:a + 1024]) for a in range(0, 4096, 1024)])
    below = np.mean(y < pred)
    assert abs(below - q) < 0.06


def test_model_bad_arguments(L):
    M = L.Model(seed=1)
    with pytest.raises(L.DSDError):
        L.dsd_model_forward(M.handle, 0, 4, 0)
    X = np.zeros((1025, 64), np.float32)
    with pytest.raises(L.DSDError):
        M.forward(X)
    with pytest.raises(L.DSDError):
        L.dsd_model_get_state(M.handle, 0, M.count)


# ------------------------------------------------------------------ features

def test_features_exact_entries_and_determinism(L, orc):
    n, s, d = gg.chung_lu(3000, 20000, 2.3, 300.0, seed=4)
    n, s, d, _ = gg.plant(n, s, d, 25, 0.8, seed=5)
    og = orc.csr(n, s, d)
    core2, _ = orc.core_decompose(og, 2)
    degen = int(core2.max())
    deg = np.diff(og.off.astype(np.int64))
    with L.Graph.from_edges(n, s, d) as g:
        for h in (2, 3, 5):
            f = g.features(h)
            assert np.array_equal(f, g.features(h))
            assert np.isclose(f[0], math.log1p(n), rtol=1e-6)
            assert np.isclose(f[1], math.log1p(og.m), rtol=1e-6)
            assert np.isclose(f[2], math.log1p(deg.max()), rtol=1e-6)
            assert np.isclose(f[3], math.log1p(degen), rtol=1e-6)
            assert np.isclose(f[4], h / 4)
            assert np.isclose(f[6], math.log1p(math.comb(degen, h - 1)), rtol=1e-4)
            assert np.isclose(f[7], math.log1p(int(np.sum(core2 == degen))), rtol=1e-6)
            assert np.isclose(f[8:24].sum(), 1, atol=1e-5)
            assert np.isclose(f[24:40].sum(), 1, atol=1e-5)
            # histogram of floor(log2(d + 1)), top bucket open
            bk = np.minimum(np.floor(np.log2(deg + 1)).astype(int), 15)
            assert np.allclose(f[8:24], np.bincount(bk, minlength=16) / n, atol=1e-6)
            # the three nested cores: V, core_2 >= degen/2, core_2 = degen
            sizes = [n, int(np.sum(2 * core2 >= degen)), int(np.sum(core2 == degen))]
            for gi, sz in enumerate(sizes):
                o = f[40 + 8 * gi: 48 + 8 * gi]
                assert np.isclose(o[0], math.log1p(sz), rtol=1e-6)
                assert 0 <= o[2] <= 1
            # inside the top core every vertex has >= degen neighbours
            assert f[57] >= math.log1p(degen) - 1e-5
            assert np.all(np.isfinite(f))


@pytest.mark.parametrize("h", [3, 4])
def test_features_on_closed_forms(L, h):
    # K_40: every sampled pair closes, each vertex lies in C(39,2) triangles
    # and C(39,h-1) h-cliques, the h-clique density is C(39,h-1)/h -- in all
    # three cores (they are all of V)
    k = 40
    s, d = zip(*[(a, b) for a in range(k) for b in range(a + 1, k)])
    with L.Graph.from_edges(k, np.array(s, np.uint32), np.array(d, np.uint32)) as g:
        f = g.features(h)
    for gi in range(3):
        o = f[40 + 8 * gi: 48 + 8 * gi]
        assert np.isclose(o[1], math.log1p(k - 1), rtol=1e-6)
        assert o[2] == 1.0
        assert np.isclose(o[3], math.log1p(math.comb(k - 1, 2)), rtol=1e-5)
        assert np.isclose(o[4], math.log1p(math.comb(k - 1, h - 1)), rtol=1e-4)
        assert np.isclose(o[5], math.log1p(math.comb(k - 1, h - 1) / h), rtol=1e-4)
    # K_{30,30}: triangle-free, so every estimate is 0
    s, d = zip(*[(a, 30 + b) for a in range(30) for b in range(30)])
    with L.Graph.from_edges(60, np.array(s, np.uint32), np.array(d, np.uint32)) as g:
        f = g.features(h)
    for gi in range(3):
        o = f[40 + 8 * gi: 48 + 8 * gi]
        assert np.isclose(o[1], math.log1p(30), rtol=1e-6)
        assert o[2] == 0 and o[3] == 0 and o[4] == 0 and o[5] == 0


# ------------------------------------------------------------- seeded path

def _const_model(L, rho_target):
    """A network whose output is the constant log1p(rho_target): all weights
    zero, b4 set."""
    M = L.Model(seed=0)
    st = np.zeros(3 * mlp.NPARAMS + 1, np.float32)
    st[mlp.NPARAMS - 1] = np.float32(np.log1p(rho_target)) if np.isfinite(rho_target) \
        else np.float32(rho_target)
    M.set_state(st)
    return M


def _expected_accept(orc, og, h, rho, core2):
    """The exact acceptance test, recomputed from the oracle: k = ceil(rho');
    accepted iff some level is >= k and the densest level >= k has density
    at least k - 1."""
    if not (math.isfinite(rho) and 0 < rho < 4.6e18):
        return False, None
    k = max(1, math.ceil(Fraction(rho)))
    degen = int(core2.max()) if len(core2) else 0
    x0 = h - 1
    while math.comb(x0, h - 1) < k and x0 <= degen:
        x0 += 1
    if x0 > degen:
        return False, (k, None)
    core, kmax = orc.core_decompose(og, h)
    lk, ls, lm = orc.level_stats(og, h, core)
    idx = [j for j in range(len(lk)) if lk[j] >= k]
    if not idx:
        return False, (k, x0)
    best = max(Fraction(int(lm[j]), int(ls[j])) for j in idx)
    return best >= k - 1, (k, x0)


def _check_seeded(L, orc, n, s, d, h, targets):
    og = orc.csr(n, s, d)
    core2, _ = orc.core_decompose(og, 2)
    wcore, wk = orc.core_decompose(og, h)
    w = orc.core_app(og, h, wcore, wk)
    lk, _, _ = orc.level_stats(og, h, wcore)
    seen = set()
    with L.Graph.from_edges(n, s, d) as g:
        for t in targets:
            M = _const_model(L, t)
            r = g.core_app_seeded(h, M)
            info = r["seed"]
            acc, kx = _expected_accept(orc, og, h, info["rho_prime"], core2)
            assert info["accepted"] == int(acc), (t, info)
            # the result record carries the same decision
            assert r["seeded_accepted"] == info["accepted"] and r["seed_k"] == info["seed_k"]
            seen.add(bool(acc))
            if kx is not None:
                assert info["seed_k"] == kx[0]
                if kx[1] is None:
                    assert info["x0"] > int(core2.max() if len(core2) else 0)
                else:
                    assert info["x0"] == kx[1]
                if acc:
                    assert info["sub_n"] == int(np.sum(core2 >= kx[1]))
            assert r["kmax"] == w["kmax"]
            assert np.array_equal(r["kmax_core"], w["kmax_core"])
            assert r["kmax_core_mu"] == w["kmax_core_mu"]
            assert r["best_k"] == w["best_k"]
            assert np.array_equal(r["densest"], w["densest"])
            assert (r["densest_mu"], r["densest_size"]) == (w["densest_mu"], w["densest_size"])
            want_levels = int(np.sum(lk >= info["seed_k"])) if acc else len(lk)
            assert r["nlevels"] == want_levels
            # the plain call on the same graph still agrees afterwards
            p = g.core_app(h)
            assert p["kmax"] == w["kmax"] and p["best_k"] == w["best_k"]
            # the boundary's seven-argument call answers the same
            rr = L.dsd_core_app_seeded(g.handle, h, M.handle, 0, 0, L.DSD_MEM_HOST)
            assert (int(rr.kmax), int(rr.best_k), int(rr.densest_mu), int(rr.densest_size),
                    int(rr.seeded_accepted), int(rr.seed_k)) == (
                w["kmax"], w["best_k"], w["densest_mu"], w["densest_size"], info["accepted"],
                info["seed_k"])
    return seen


@pytest.mark.parametrize("h", [2, 3, 4])
def test_seeded_equals_plain(L, orc, h):
    n, s, d = gg.chung_lu(4000, 30000, 2.2, 400.0, seed=10 + h)
    n, s, d, _ = gg.plant(n, s, d, 30, 0.7, seed=20 + h)
    og = orc.csr(n, s, d)
    wcore, wk = orc.core_decompose(og, h)
    w = orc.core_app(og, h, wcore, wk)
    rho_opt = w["densest_mu"] / w["densest_size"]
    targets = [0.0, 0.3, 0.5 * rho_opt, 0.9 * rho_opt, rho_opt * 0.999, rho_opt * 1.05,
               float(wk) + 0.5, 10 * rho_opt + 100, 1e30, float("nan"), float("inf")]
    seen = _check_seeded(L, orc, n, s, d, h, targets)
    assert seen == {True, False}


def test_seeded_small_and_degenerate(L, orc):
    # empty graph, no edges, one clique, a clique below h
    cases = [
        (1, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3),
        (5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3),
        (6,) + tuple(np.array(e, np.uint32) for e in zip(*[(a, b) for a in range(6)
                                                           for b in range(a + 1, 6)])) + (4,),
        (3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), 3),
    ]
    for n, s, d, h in cases:
        _check_seeded(L, orc, n, s, d, h, [0.5, 1.0, 2.0, 7.0, 1e6])


def test_seeded_random_graphs(L, orc):
    r = np.random.default_rng(44)
    for it in range(12):
        n, s, d = gg.random_small(int(r.integers(20, 300)), float(r.uniform(0.02, 0.3)),
                                  seed=int(r.integers(1 << 30)))
        h = int(r.integers(2, 6))
        _check_seeded(L, orc, n, s, d, h, [float(r.uniform(0, 20)), float(r.uniform(0, 3))])


def test_seeded_rejects_bad_arguments(L):
    n, s, d = gg.er(100, 0.1, seed=1)
    M = L.Model(seed=0)
    with L.Graph.from_edges(n, s, d) as g:
        with pytest.raises(L.DSDError):
            L.dsd_core_app_seeded(g.handle, 1, M.handle, 0, 0, L.DSD_MEM_HOST)
        with pytest.raises(L.DSDError):
            L.dsd_core_app_seeded(g.handle, 3, 0, 0, 0, L.DSD_MEM_HOST)


# ---------------------------------------------------------------- training

def test_training_labels_match_oracle(L, orc):
    # a 5% sample of the first 400 training graphs (those the oracle finishes
    # quickly): the label's densest level equals the oracle's exactly
    from paper_1906_00341_gb300 import train
    checked = 0
    for i in range(0, 400, 20):
        n, s, d, h = gg.train_graph(i)
        if n > 20000:
            continue
        f, lab, (mu, size), m = train.label_graph(n, s, d, h)
        og = orc.csr(n, s, d)
        w = orc.core_app(og, h)
        assert (mu, size) == (w["densest_mu"], w["densest_size"]), i
        assert math.isclose(lab, math.log1p(mu / size), rel_tol=1e-6)
        assert m == og.m
        checked += 1
    assert checked >= 10


def test_checkpoint_roundtrip(L, tmp_path):
    from paper_1906_00341_gb300 import train
    r = np.random.default_rng(1)
    X = r.standard_normal((600, 64)).astype(np.float32)
    y = (X[:, 1] * 0.5 + 3).astype(np.float32)
    M, hist = train.train(X, y, epochs=3, log=None)
    assert len(hist) == 3 and "val_below" in hist[-1]
    p = tmp_path / "m.npz"
    train.save_checkpoint(M, str(p), 3, dict(note="test"))
    M2 = train.load_checkpoint(str(p))
    assert np.array_equal(M2.state(), M.state())
    assert np.array_equal(train.predict(M2, X), train.predict(M, X))
    # a corrupted state is refused
    with np.load(str(p)) as z:
        st, hd = z["state"].copy(), z["header"]
    st[5] += 1
    bad = tmp_path / "bad.npz"
    np.savez(str(bad), state=st, header=hd)
    with pytest.raises(ValueError):
        train.load_checkpoint(str(bad))


# ------------------------------------------------- CoreApp's top-down schedule

def _check_topdown(L, orc, n, s, d, h):
    og = orc.csr(n, s, d)
    wcore, wk = orc.core_decompose(og, h)
    w = orc.core_app(og, h, wcore, wk)
    lk, _, _ = orc.level_stats(og, h, wcore)
    core2, _ = orc.core_decompose(og, 2)
    with L.Graph.from_edges(n, s, d) as g:
        r = g.core_app_topdown(h)
    sc = r["schedule"]
    assert r["kmax"] == w["kmax"]
    assert np.array_equal(r["kmax_core"], w["kmax_core"])
    assert r["kmax_core_mu"] == w["kmax_core_mu"]
    assert r["best_k"] == w["best_k"]
    assert np.array_equal(r["densest"], w["densest"])
    assert (r["densest_mu"], r["densest_size"]) == (w["densest_mu"], w["densest_size"])
    assert sc["passes"] >= 1 and sc["sub_n"] <= n
    if h > 2 and n:
        # the last window is the edge core {core_2 >= x}; gamma_out is the
        # largest C(core_2, h-1) outside it, and every core >= k_max sits inside
        assert sc["sub_n"] == int(np.sum(core2 >= sc["x"]))
        outside = core2[core2 < sc["x"]]
        g_out = math.comb(int(outside.max()), h - 1) if outside.size else 0
        assert sc["gamma_out"] == g_out
        assert w["kmax"] > g_out or sc["sub_n"] == n
        assert r["nlevels"] == int(np.sum(lk >= g_out + 1)) or sc["sub_n"] == n
    return sc


@pytest.mark.parametrize("h", [3, 4, 5])
def test_topdown_equals_plain(L, orc, h):
    n, s, d = gg.chung_lu(6000, 40000, 2.2, 500.0, seed=30 + h)
    n, s, d, _ = gg.plant(n, s, d, 40, 0.7, seed=40 + h)
    sc = _check_topdown(L, orc, n, s, d, h)
    assert sc["sub_n"] < n   # the schedule stopped before the whole graph


def test_topdown_small_and_random(L, orc):
    _check_topdown(L, orc, 1, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3)
    _check_topdown(L, orc, 9, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3)
    r = np.random.default_rng(7)
    for it in range(10):
        n, s, d = gg.random_small(int(r.integers(20, 400)), float(r.uniform(0.02, 0.3)),
                                  seed=int(r.integers(1 << 30)))
        _check_topdown(L, orc, n, s, d, int(r.integers(2, 6)))


# ---------------------------------------------- what the trained network gains

def test_trained_proposal_narrows_the_work(L, orc):
    """A held-out graph (Chung-Lu with planted blocks, the evaluation
    workload's shape, seeds never used in training): the trained checkpoint's
    proposal is accepted and leaves only a small edge core to decompose,
    while an untrained network of the same architecture (He-uniform weights)
    and the method without a proposal (the plain path) decompose far more of
    the graph; every answer equals the oracle's."""
    from paper_1906_00341_gb300 import train
    n, s, d, h = gg.heldout_graph(15)
    M = train.load_checkpoint(train.DEFAULT_CHECKPOINT)
    U = L.Model(seed=1)
    og = orc.csr(n, s, d)
    wcore, wk = orc.core_decompose(og, h)
    w = orc.core_app(og, h, wcore, wk)
    with L.Graph.from_edges(n, s, d) as g:
        rt = g.core_app_seeded(h, M)
        ru = g.core_app_seeded(h, U)
        rp = g.core_app(h)
    for r in (rt, ru, rp):
        assert r["kmax"] == w["kmax"] and r["best_k"] == w["best_k"]
        assert np.array_equal(r["kmax_core"], w["kmax_core"])
        assert np.array_equal(r["densest"], w["densest"])
        assert (r["densest_mu"], r["densest_size"]) == (w["densest_mu"], w["densest_size"])
    assert rt["seed"]["accepted"] == 1
    # vertices each call decomposes: the accepted edge core, else all of G
    def work(r):
        return r["seed"]["sub_n"] if r["seed"]["accepted"] else n
    assert work(rt) * 20 <= n
    assert work(rt) * 4 <= work(ru)
