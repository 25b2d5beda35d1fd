"""Pins of the exact CDS oracle (Algorithm 1, Sec. 3.1) against facts it
does not compute itself:

* brute force over all vertex subsets (n <= 12): rho_opt is the largest
  mu(S)/|S|, and the returned set is the union of every subset reaching it;
* an independent exact search (Dinkelbach's iteration on the same networks,
  Python integers, tests/flow.py) on graphs too large for brute force;
* closed forms: K_n, two disjoint equal cliques (both are returned), a
  larger and a smaller clique (the larger alone), K_{a,b} at h = 2, a clique
  with a pendant path;
* the paper's facts about the optimum: the CDS lies in the
  (ceil(rho_opt), Psi)-core (Sec. 4.3 lemma used by CoreExact), each of its
  vertices lies in at least rho_opt of its cliques (removing a vertex never
  raises the density of a densest set), and rho(S*) <= rho_opt <= k_max,
  rho(R_kmax) >= rho_opt / h (Lemma 3, Lemma 6).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as bf
import flow
from paper_1906_00341_gb300 import graphgen as gg


def _graph(orc, n, pairs):
    pairs = np.asarray(pairs, np.uint32).reshape(-1, 2)
    return orc.csr(n, pairs[:, 0].copy(), pairs[:, 1].copy())


def _clique_pairs(verts):
    return [(a, b) for i, a in enumerate(verts) for b in verts[i + 1:]]


def _brute(A, h):
    """(rho_opt, union of all maximisers) over non-empty subsets."""
    n = A.shape[0]
    subsets, inS, _, muS = bf._subset_tables(A, h)
    size = inS.sum(1)
    best = Fraction(0)
    for S in range(1, 1 << n):
        f = Fraction(int(muS[S]), int(size[S]))
        if f > best:
            best = f
    union = np.zeros(n, bool)
    for S in range(1, 1 << n):
        if Fraction(int(muS[S]), int(size[S])) == best:
            union |= inS[S]
    return best, np.flatnonzero(union)


@pytest.mark.parametrize("h", [2, 3, 4])
def test_exact_bruteforce(orc, h):
    rng = np.random.default_rng(4242 + h)
    for i in range(14):
        n = int(rng.integers(2, 13))
        p = float(rng.choice([0.3, 0.5, 0.7, 0.85]))
        n, s, d = gg.random_small(n, p, seed=6000 + 31 * h + i)
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        r = orc.exact_cds(g, h)
        best, union = _brute(A, h)
        if best == 0:
            assert r["mu"] == 0 and r["size"] == n and r["cds"].size == n
            continue
        assert Fraction(r["mu"], r["size"]) == best, (n, h, i)
        assert np.array_equal(r["cds"], union), (n, h, i, r["cds"], union)
        assert r["size"] == r["cds"].size
        assert r["mu"] == orc.induced_clique_count(g, h, np.isin(np.arange(n), r["cds"]))
        # one cut as a certificate: nothing beats rho_opt, and just below it
        # something does
        beats, side = orc.densest_check(g, h, best.numerator, best.denominator)
        assert not beats and np.array_equal(side, union)
        below = best - Fraction(1, 1000 * n * n)
        assert orc.densest_check(g, h, below.numerator, below.denominator)[0]


def test_exact_matches_dinkelbach(orc):
    rng = np.random.default_rng(99)
    for i in range(6):
        n = int(rng.integers(18, 34))
        n, s, d = gg.random_small(n, float(rng.choice([0.2, 0.35, 0.5])), seed=7100 + i)
        if i % 2:
            n, s, d, _ = gg.plant(n, s, d, 9, 0.9, 7200 + i)
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        for h in (2, 3, 4):
            r = orc.exact_cds(g, h)
            rho, _ = flow.rho_opt(A, h)
            if rho == 0:
                assert r["mu"] == 0
            else:
                assert Fraction(r["mu"], r["size"]) == rho, (i, h)


@pytest.mark.parametrize("h", [2, 3, 4])
def test_exact_closed_forms(orc, h):
    # K_n: the whole clique, C(n, h) / n
    for n in (5, 7):
        g = _graph(orc, n, _clique_pairs(list(range(n))))
        r = orc.exact_cds(g, h)
        assert r["size"] == n and Fraction(r["mu"], r["size"]) == Fraction(math.comb(n, h), n)
    # two disjoint K_6: both reach the optimum, the union is returned
    pairs = _clique_pairs(list(range(6))) + _clique_pairs(list(range(6, 12)))
    r = orc.exact_cds(_graph(orc, 14, pairs + [(12, 13)]), h)
    assert r["cds"].tolist() == list(range(12))
    assert r["mu"] == 2 * math.comb(6, h)
    # K_7 beside K_5: the larger clique alone
    pairs = _clique_pairs(list(range(7))) + _clique_pairs(list(range(7, 12)))
    r = orc.exact_cds(_graph(orc, 12, pairs), h)
    assert r["cds"].tolist() == list(range(7))
    # K_6 with a pendant path 5-6-7-8-9: the clique alone
    pairs = _clique_pairs(list(range(6))) + [(5, 6), (6, 7), (7, 8), (8, 9)]
    r = orc.exact_cds(_graph(orc, 10, pairs), h)
    assert r["cds"].tolist() == list(range(6))
    assert Fraction(r["mu"], r["size"]) == Fraction(math.comb(6, h), 6)


def test_exact_bipartite_and_empty(orc):
    # K_{a,b} at h = 2: every subgraph K_{x,y} has density xy/(x+y), largest
    # at the whole graph
    a, b = 3, 5
    g = _graph(orc, a + b, [(i, a + j) for i in range(a) for j in range(b)])
    r = orc.exact_cds(g, 2)
    assert r["size"] == a + b and Fraction(r["mu"], r["size"]) == Fraction(a * b, a + b)
    # no triangle in K_{a,b}: density 0 everywhere, the answer is V
    r = orc.exact_cds(g, 3)
    assert r["mu"] == 0 and r["cds"].tolist() == list(range(a + b))
    # edgeless graph
    r = orc.exact_cds(orc.csr(4, np.zeros(0, np.uint32), np.zeros(0, np.uint32)), 2)
    assert r["mu"] == 0 and r["size"] == 4


@pytest.mark.parametrize("h", [2, 3, 4])
def test_exact_lemmas(orc, h):
    for seed in range(4):
        n, s, d = gg.er(160, 0.05, 7300 + seed)
        n, s, d, _ = gg.plant(n, s, d, 14 + 2 * seed, 0.7, 7400 + seed)
        g = orc.csr(n, s, d)
        r = orc.exact_cds(g, h)
        rho = Fraction(r["mu"], r["size"])
        core, kmax = orc.core_decompose(g, h)
        # the CDS lies in the (ceil(rho_opt), Psi)-core
        k = math.ceil(rho)
        assert np.all(core[r["cds"]] >= k)
        # each CDS vertex is in >= rho_opt cliques of the CDS
        mask = np.zeros(n, bool)
        mask[r["cds"]] = True
        sub = orc.csr(n, *_induced_pairs(g, mask))
        deg, mu = orc.clique_degrees(sub, h)
        assert mu == r["mu"]
        assert all(Fraction(int(deg[v])) >= rho for v in r["cds"])
        # Lemma 3 / Lemma 6 and the densest level
        app = orc.core_app(g, h, core, kmax)
        assert rho <= kmax
        assert Fraction(app["kmax_core_mu"], app["kmax_core"].size) >= rho / h
        assert Fraction(app["densest_mu"], app["densest_size"]) <= rho


def _induced_pairs(g, mask):
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.off).astype(np.int64))
    keep = mask[src] & mask[g.adj] & (src < g.adj)
    return src[keep].copy(), g.adj[keep].copy()
