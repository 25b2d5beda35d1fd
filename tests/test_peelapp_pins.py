"""Pins of the oracle's PeelApp (Algorithm 2) against facts it does not
compute itself:

* a direct simulation on small graphs with Python sets and brute-force clique
  counts (remove a vertex of least current clique-degree, smaller id first;
  keep the first strictly densest set, starting from G);
* Lemma 2: rho(S*) >= rho_opt / h, with rho_opt from brute force or the
  exact oracle;
* a minimum-degree peel passes through every (k,Psi)-core R_k (while the
  current set strictly contains R_k, some vertex outside R_k has fewer than
  k cliques in it), so rho(S*) >= max_k rho(R_k), the CoreApp density;
* closed forms: K_n returns K_n; a larger and a smaller disjoint clique
  return the larger one.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as bf
from paper_1906_00341_gb300 import graphgen as gg


def _simulate(A, h):
    n = A.shape[0]
    alive = set(range(n))

    def count_in(S):
        return sum(1 for c in itertools.combinations(sorted(S), h)
                   if all(A[a, b] for a, b in itertools.combinations(c, 2)))

    def deg_in(S, v):
        others = sorted(S - {v})
        return sum(1 for c in itertools.combinations(others, h - 1)
                   if all(A[v, x] for x in c) and all(A[a, b] for a, b in itertools.combinations(c, 2)))

    best_set, best = set(alive), Fraction(count_in(alive), n) if n else Fraction(0)
    order = []
    while alive:
        v = min(alive, key=lambda x: (deg_in(alive, x), x))
        order.append(v)
        alive.remove(v)
        if alive:
            d = Fraction(count_in(alive), len(alive))
            if d > best:
                best, best_set = d, set(alive)
    return best_set, best, order


@pytest.mark.parametrize("h", [2, 3, 4])
def test_peelapp_simulation(orc, h):
    rng = np.random.default_rng(9600 + h)
    for i in range(10):
        n = int(rng.integers(3, 13))
        n, s, d = gg.random_small(n, float(rng.choice([0.3, 0.5, 0.7])), seed=9700 + 13 * h + i)
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        r = orc.peel_app(g, h)
        want_set, want, want_order = _simulate(A, h)
        assert r["set"].tolist() == sorted(want_set), (h, i)
        assert Fraction(r["mu"], r["size"]) == want
        # the whole removal order, ties to the smaller id
        assert np.asarray(r["order"]).tolist() == want_order, (h, i)
        # Lemma 2 against brute force
        rho_opt = bf.rho_opt(A, h)
        assert Fraction(r["mu"], r["size"]) >= rho_opt / h


@pytest.mark.parametrize("h", [2, 3, 4])
def test_peelapp_levels_and_lemma2(orc, h):
    for seed in range(3):
        n, s, d = gg.er(200, 0.05, 9800 + seed)
        n, s, d, _ = gg.plant(n, s, d, 16, 0.8, 9900 + seed)
        g = orc.csr(n, s, d)
        r = orc.peel_app(g, h)
        rho = Fraction(r["mu"], r["size"])
        assert r["mu"] == orc.induced_clique_count(g, h, np.isin(np.arange(n), r["set"]))
        assert r["size"] == r["set"].size
        app = orc.core_app(g, h)
        assert rho >= Fraction(app["densest_mu"], app["densest_size"])
        ex = orc.exact_cds(g, h)
        assert rho <= Fraction(ex["mu"], ex["size"])
        assert rho >= Fraction(ex["mu"], ex["size"]) / h


def test_peelapp_closed_forms(orc):
    for h in (2, 3, 4):
        n = 7
        s, d = np.triu_indices(n, 1)
        r = orc.peel_app(orc.csr(n, s.astype(np.uint32), d.astype(np.uint32)), h)
        assert r["set"].tolist() == list(range(n)) and r["mu"] == math.comb(n, h)
        pairs = [(a, b) for a in range(6) for b in range(a + 1, 6)] + \
                [(a, b) for a in range(6, 10) for b in range(a + 1, 10)]
        p = np.array(pairs, np.uint32)
        r = orc.peel_app(orc.csr(10, p[:, 0].copy(), p[:, 1].copy()), h)
        assert r["set"].tolist() == list(range(6))
    # no triangle: the whole graph, density 0
    r = orc.peel_app(orc.csr(4, np.array([0, 1, 2], np.uint32), np.array([1, 2, 3], np.uint32)), 3)
    assert r["mu"] == 0 and r["size"] == 4


@pytest.mark.parametrize("h", [2, 3, 4])
def test_peelapp_removes_the_levels_in_order(orc, h):
    """The fact the GPU's per-level PeelApp rests on: the one-at-a-time peel
    removes every vertex of core number k before any of core number k + 1
    (the minimum is always taken outside R_{k+1}), so its removal order is
    sorted by the (k,Psi)-core numbers of Algorithm 3."""
    for seed in range(4):
        n, s, d = gg.er(150, 0.06 + 0.02 * seed, 9950 + seed)
        n, s, d, _ = gg.plant(n, s, d, 14, 0.8, 9960 + seed)
        g = orc.csr(n, s, d)
        order = np.asarray(orc.peel_app(g, h)["order"], np.int64)
        core, _ = orc.core_decompose(g, h)
        assert sorted(order.tolist()) == list(range(n))
        assert np.all(np.diff(np.asarray(core, np.int64)[order]) >= 0), (h, seed)
