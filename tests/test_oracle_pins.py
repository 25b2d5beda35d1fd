"""Pins for the CPU oracle: checks against things other than itself.

* brute force over all vertex subsets (n <= 16) of the definitions;
* closed forms (K_n, disjoint cliques, stars, cycles, complete bipartite,
  the empty graph);
* the paper's worked examples under tests/golden/;
* identities: sum of clique-degrees = h * mu; h = 2 gives the degree;
  h = 3 gives diag(A^3)/2 (dense matrix product);
* invariants: core <= clique-degree (Sec. 4.1), the gamma bound
  core(v) <= C(core_2(v), h-1) (Sec. 5.2), Theorem 1, Lemma 3 and Lemma 6
  against an exact min-cut rho_opt, tie-order independence of Algorithm 3,
  the threshold-pruning certificate of every level.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as bf
import flow
from paper_1906_00341_gb300 import graphgen as gg

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def graph_from_pairs(orc, n, pairs):
    pairs = np.asarray(pairs, np.uint32).reshape(-1, 2)
    return orc.csr(n, pairs[:, 0].copy(), pairs[:, 1].copy())


def complete(orc, n):
    s, d = np.triu_indices(n, 1)
    return orc.csr(n, s.astype(np.uint32), d.astype(np.uint32))


def small_graphs(count=24, nmax=14):
    rng = np.random.default_rng(12345)
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        p = float(rng.choice([0.2, 0.4, 0.6, 0.8]))
        yield gg.random_small(n, p, seed=1000 + i)


def read_golden(name):
    meta, edges, in_edges = {}, [], False
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line == "edges:":
                in_edges = True
                continue
            if in_edges:
                a, b = line.split()
                edges.append((int(a), int(b)))
            else:
                k, v = line.split(":", 1)
                meta[k.strip()] = v.strip()
    return meta, edges


def parse_map(s):
    return {int(a): int(b) for a, b in (t.split("=") for t in s.split())}


# ----------------------------------------------------------------- CSR ---

def test_csr_matches_set_construction(orc):
    for n, s, d in small_graphs(12, 20):
        g = orc.csr(n, s, d)
        want = [set() for _ in range(n)]
        for a, b in zip(s.tolist(), d.tolist()):
            if a != b:
                want[a].add(b)
                want[b].add(a)
        for v in range(n):
            row = g.adj[g.off[v]:g.off[v + 1]].tolist()
            assert row == sorted(want[v])


def test_csr_rejects_out_of_range(orc):
    with pytest.raises(ValueError):
        orc.csr(3, np.array([0, 3], np.uint32), np.array([1, 1], np.uint32))


# ------------------------------------------------------ clique-degrees ---

@pytest.mark.parametrize("h", [2, 3, 4, 5])
def test_clique_degrees_bruteforce(orc, h):
    for n, s, d in small_graphs():
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        want, wmu = bf.clique_degrees(A, h)
        got, mu = orc.clique_degrees(g, h)
        assert mu == wmu
        assert got.astype(np.int64).tolist() == want.tolist()


@pytest.mark.parametrize("n", [1, 2, 5, 9, 13])
@pytest.mark.parametrize("h", [2, 3, 4, 6])
def test_complete_graph_closed_form(orc, n, h):
    g = complete(orc, n)
    deg, mu = orc.clique_degrees(g, h)
    assert mu == math.comb(n, h)
    assert set(deg.tolist()) == {math.comb(n - 1, h - 1)}
    core, kmax = orc.core_decompose(g, h)
    assert set(core.tolist()) == {math.comb(n - 1, h - 1)}
    assert kmax == math.comb(n - 1, h - 1)
    res = orc.core_app(g, h)
    assert res["kmax_core"].tolist() == list(range(n))
    assert Fraction(res["densest_mu"], res["densest_size"]) == Fraction(math.comb(n, h), n)


def test_sum_identity_and_degree(orc):
    for n, s, d in small_graphs(10, 40):
        g = orc.csr(n, s, d)
        for h in (2, 3, 4):
            deg, mu = orc.clique_degrees(g, h)
            assert int(deg.sum()) == h * mu
        deg2, mu2 = orc.clique_degrees(g, 2)
        assert deg2.tolist() == g.degree().tolist()
        assert mu2 == g.m


def test_triangles_match_matrix_cube(orc):
    n, s, d = gg.er(400, 0.05, 3)
    g = orc.csr(n, s, d)
    A = np.zeros((n, n), np.int64)
    for v in range(n):
        A[v, g.adj[g.off[v]:g.off[v + 1]]] = 1
    want = np.diag(A @ A @ A) // 2
    got, mu = orc.clique_degrees(g, 3)
    assert got.astype(np.int64).tolist() == want.tolist()
    assert mu == int(np.trace(A @ A @ A)) // 6


def test_vertex_clique_degree(orc):
    n, s, d = gg.er(300, 0.08, 4)
    g = orc.csr(n, s, d)
    for h in (3, 4):
        deg, _ = orc.clique_degrees(g, h)
        for v in (0, 17, 150, 299):
            assert orc.vertex_clique_degree(g, h, v) == int(deg[v])


def test_golden_two_triangles(orc):
    meta, edges = read_golden("def3_two_triangles_h3.txt")
    g = graph_from_pairs(orc, int(meta["n"]), edges)
    deg, mu = orc.clique_degrees(g, int(meta["h"]))
    assert mu == int(meta["mu"])
    for v, want in parse_map(meta["clique_degree"]).items():
        assert int(deg[v]) == want


def test_golden_example3_k4(orc):
    meta, edges = read_golden("ex3_k4_h3.txt")
    g = graph_from_pairs(orc, int(meta["n"]), edges)
    h = int(meta["h"])
    deg, mu = orc.clique_degrees(g, h)
    assert mu == int(meta["mu"])
    assert {v: int(deg[v]) for v in range(4)} == parse_map(meta["clique_degree"])
    core, kmax = orc.core_decompose(g, h)
    assert {v: int(core[v]) for v in range(4)} == parse_map(meta["core"])
    assert kmax == int(meta["kmax"])


def test_golden_example4_bounds(orc):
    meta, _ = read_golden("ex4_bounds_h2.txt")
    assert meta["family_density"] == "(1+4x)/(2+2x)"
    c4 = graph_from_pairs(orc, 4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    r = orc.core_app(c4, 2)
    assert r["kmax"] == int(meta["cycle4_kmax"])
    assert (r["kmax_core_mu"], r["kmax_core"].size) == (4, 4)   # density 4/4
    for x in range(1, 7):
        n = 2 + 2 * x
        pairs = [(0, 1)]
        for i in range(x):
            c, dd = 2 + 2 * i, 3 + 2 * i
            pairs += [(0, c), (1, c), (0, dd), (1, dd)]
        g = graph_from_pairs(orc, n, pairs)
        r = orc.core_app(g, 2)
        assert r["kmax"] == int(meta["family_kmax"])
        assert Fraction(r["kmax_core_mu"], r["kmax_core"].size) == Fraction(1 + 4 * x, 2 + 2 * x)


# ----------------------------------------------------- core numbers ------

@pytest.mark.parametrize("h", [2, 3, 4])
def test_core_bruteforce(orc, h):
    for n, s, d in small_graphs(20, 13):
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        want = bf.core_numbers(A, h)
        core, kmax = orc.core_decompose(g, h)
        assert core.astype(np.int64).tolist() == want.tolist()
        assert kmax == (int(want.max()) if n else 0)


def test_core_tie_order_independent(orc):
    for i, name in enumerate(["er", "cl"]):
        if name == "er":
            n, s, d = gg.er(500, 0.03, 10 + i)
        else:
            n, s, d = gg.chung_lu(2000, 12000, 2.3, 200.0, 11)
        g = orc.csr(n, s, d)
        for h in (2, 3, 4):
            a, ka = orc.core_decompose(g, h, 0)
            b, kb = orc.core_decompose(g, h, 1)
            assert ka == kb and a.tolist() == b.tolist()


def test_closed_form_families(orc):
    # disjoint K_a + K_b
    a, b = 6, 9
    pairs = [(i, j) for i, j in itertools.combinations(range(a), 2)]
    pairs += [(a + i, a + j) for i, j in itertools.combinations(range(b), 2)]
    g = graph_from_pairs(orc, a + b, pairs)
    for h in (2, 3, 4):
        core, kmax = orc.core_decompose(g, h)
        assert core[:a].tolist() == [math.comb(a - 1, h - 1)] * a
        assert core[a:].tolist() == [math.comb(b - 1, h - 1)] * b
        r = orc.core_app(g, h)
        assert r["kmax_core"].tolist() == list(range(a, a + b))
    # star K_{1,s}: h=2 cores all 1; no triangles
    s_ = 11
    g = graph_from_pairs(orc, s_ + 1, [(0, i) for i in range(1, s_ + 1)])
    core, kmax = orc.core_decompose(g, 2)
    assert set(core.tolist()) == {1} and kmax == 1
    core, kmax = orc.core_decompose(g, 3)
    assert set(core.tolist()) == {0} and kmax == 0
    r = orc.core_app(g, 3)       # no instance: R_0 = V, density 0
    assert r["kmax_core"].size == s_ + 1 and r["densest_mu"] == 0
    # cycles
    for L in (4, 7, 12):
        g = graph_from_pairs(orc, L, [(i, (i + 1) % L) for i in range(L)])
        assert set(orc.core_decompose(g, 2)[0].tolist()) == {2}
        assert set(orc.core_decompose(g, 3)[0].tolist()) == {0}
    # complete bipartite K_{p,q}: edge core = min(p, q), triangle-free
    p_, q_ = 4, 7
    g = graph_from_pairs(orc, p_ + q_, [(i, p_ + j) for i in range(p_) for j in range(q_)])
    assert set(orc.core_decompose(g, 2)[0].tolist()) == {min(p_, q_)}
    assert orc.clique_degrees(g, 3)[1] == 0
    # empty graph
    g = orc.csr(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    core, kmax = orc.core_decompose(g, 3)
    assert core.tolist() == [0] * 5 and kmax == 0
    r = orc.core_app(g, 3)
    assert r["densest"].size == 5 and r["densest_mu"] == 0


def _invariants(orc, g, h):
    deg, mu = orc.clique_degrees(g, h)
    core, kmax = orc.core_decompose(g, h)
    core2, _ = orc.core_decompose(g, 2)
    # core <= clique-degree (Sec. 4.1, property 3)
    assert np.all(core <= deg)
    # gamma bound (Sec. 5.2): core(v) <= C(core_2(v), h-1)
    for v in range(g.n):
        assert int(core[v]) <= math.comb(int(core2[v]), h - 1)
    levels, size, lmu = orc.level_stats(g, h, core)
    for j, k in enumerate(levels.tolist()):
        mask = core >= k
        # certificate: R_k by threshold pruning equals {core >= k}
        assert np.array_equal(orc.threshold_prune(g, h, k), mask)
        # level stats vs an independent induced count
        assert int(size[j]) == int(mask.sum())
        assert int(lmu[j]) == orc.induced_clique_count(g, h, mask)
        # Theorem 1: k/h <= rho(R_k) <= kmax
        rho = Fraction(int(lmu[j]), int(size[j]))
        assert Fraction(k, h) <= rho <= kmax
    # one more level above kmax is empty
    assert not orc.threshold_prune(g, h, kmax + 1).any()
    return core, kmax


def test_invariants_random(orc):
    for i, (n, s, d) in enumerate(small_graphs(8, 60)):
        g = orc.csr(n, s, d)
        for h in (2, 3, 4):
            _invariants(orc, g, h)
    n, s, d, _ = gg.plant(300, *gg.chung_lu(300, 1500, 2.2, 60.0, 5)[1:], 25, 0.6, 6)
    g = orc.csr(n, s, d)
    for h in (2, 3, 4, 5):
        _invariants(orc, g, h)


# -------------------------------------------- rho_opt, Lemmas 3 and 6 ---

def test_flow_matches_bruteforce(orc):
    for n, s, d in small_graphs(14, 11):
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        for h in (2, 3, 4):
            r_flow, _ = flow.rho_opt(A, h)
            assert r_flow == bf.rho_opt(A, h)


def test_lemma3_lemma6_guarantee(orc):
    rng = np.random.default_rng(77)
    cases = []
    for i in range(6):
        n = int(rng.integers(12, 30))
        cases.append(gg.random_small(n, float(rng.choice([0.25, 0.4, 0.6])), 500 + i))
    cases.append(gg.plant(28, *gg.er(28, 0.15, 9)[1:], 8, 0.9, 10)[:3])
    for n, s, d in cases:
        g = orc.csr(n, s, d)
        A = bf.adjacency(n, g.off, g.adj)
        for h in (2, 3, 4):
            ropt, _ = flow.rho_opt(A, h)
            r = orc.core_app(g, h)
            if r["kmax"] == 0:
                assert ropt == 0
                continue
            kcore_rho = Fraction(r["kmax_core_mu"], r["kmax_core"].size)
            best_rho = Fraction(r["densest_mu"], r["densest_size"])
            assert ropt <= r["kmax"]                     # Lemma 3
            assert kcore_rho >= ropt / h                 # Lemma 6
            assert best_rho <= ropt                      # a feasible subgraph
            assert best_rho >= kcore_rho                 # S* is the densest level


def test_densest_level_is_argmax(orc):
    """S* is the densest of the nested level sets (ties to the larger k),
    checked against a direct scan of all thresholds k = 0..kmax."""
    n, s, d, _ = gg.plant(200, *gg.er(200, 0.04, 21)[1:], 20, 0.7, 22)
    g = orc.csr(n, s, d)
    for h in (2, 3, 4):
        core, kmax = orc.core_decompose(g, h)
        r = orc.core_app(g, h, core, kmax)
        best = None
        for k in range(0, kmax + 1):
            mask = orc.threshold_prune(g, h, k)
            rho = Fraction(orc.induced_clique_count(g, h, mask), int(mask.sum()))
            if best is None or rho >= best[0]:
                best = (rho, k, mask)
        assert Fraction(r["densest_mu"], r["densest_size"]) == best[0]
        assert r["densest"].tolist() == np.nonzero(best[2])[0].tolist()


def test_vertex_clique_degrees_batch_matches_single(orc):
    # the batched per-vertex count shares one listing order; it must agree
    # with the single-vertex call and with the full clique-degree vector
    import numpy as np
    from paper_1906_00341_gb300 import graphgen as gg
    n, s, d = gg.random_small(120, 0.15, seed=11)
    g = orc.csr(n, s, d)
    for h in (2, 3, 4):
        full, _ = orc.clique_degrees(g, h)
        vs = np.array([0, 5, 17, 17, 119, 64], np.uint32)
        got = orc.vertex_clique_degrees(g, h, vs)
        assert np.array_equal(got, full[vs])
        assert [orc.vertex_clique_degree(g, h, int(v)) for v in vs] == got.tolist()
