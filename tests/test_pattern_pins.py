"""Pins of the pattern oracle (Sec. 6: pattern instances, pattern-degree,
(k, Psi)-cores for the x-star and the 4-vertex loop) against brute force and
closed forms it does not compute itself."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

from paper_1906_00341_gb300 import graphgen as gg


def _adj_sets(n, s, d):
    A = [set() for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            A[a].add(b)
            A[b].add(a)
    return A


def _instances(A, nodes, pattern, x):
    """Every instance as a frozenset of vertices (with multiplicity: distinct
    edge sets on the same vertices are distinct instances)."""
    out = []
    nodes = sorted(nodes)
    S = set(nodes)
    if pattern == "star":
        for c in nodes:
            for leaves in itertools.combinations(sorted(A[c] & S), x):
                out.append(frozenset((c,) + leaves))
    else:
        for q in itertools.combinations(nodes, 4):
            a, b, c, d = q
            for cyc in ((a, b, c, d), (a, b, d, c), (a, c, b, d)):
                if all(cyc[(i + 1) % 4] in A[cyc[i]] for i in range(4)):
                    out.append(frozenset(q))
    return out


def _brute_degrees(A, nodes, pattern, x, n):
    deg = np.zeros(n, np.int64)
    inst = _instances(A, nodes, pattern, x)
    for I in inst:
        for v in I:
            deg[v] += 1
    return deg, len(inst)


PATTERNS = [("star", 2), ("star", 3), ("loop", 0)]


def _code(orc, name):
    return orc.STAR if name == "star" else orc.LOOP4


@pytest.mark.parametrize("name,x", PATTERNS)
def test_pattern_degrees_brute_force(orc, name, x):
    for seed in range(12):
        n, s, d = gg.random_small(9 + seed % 4, 0.3 + 0.05 * (seed % 5), seed=500 + seed)
        A = _adj_sets(n, s, d)
        g = orc.csr(n, s, d)
        deg, mu = orc.pattern_degrees(g, _code(orc, name), x)
        want, wmu = _brute_degrees(A, range(n), name, x, n)
        assert mu == wmu and np.array_equal(deg.astype(np.int64), want)
        # sum of pattern-degrees = |V_Psi| mu
        assert int(deg.sum()) == orc.pattern_size(_code(orc, name), x) * mu


def test_pattern_closed_forms(orc):
    # K_n: C(n,4) vertex sets, 3 loops each; x-stars: n C(n-1, x)
    for n in (4, 5, 7):
        s, d = np.triu_indices(n, 1)
        g = orc.csr(n, s.astype(np.uint32), d.astype(np.uint32))
        deg, mu = orc.pattern_degrees(g, orc.LOOP4)
        assert mu == 3 * math.comb(n, 4) and set(deg.tolist()) == {3 * math.comb(n - 1, 3)}
        for x in (2, 3):
            deg, mu = orc.pattern_degrees(g, orc.STAR, x)
            assert mu == n * math.comb(n - 1, x)
            assert set(deg.tolist()) == {math.comb(n - 1, x) + (n - 1) * math.comb(n - 2, x - 1)}
    # K_{a,b}: every 2 + 2 choice is one loop
    a, b = 4, 5
    s = np.repeat(np.arange(a), b).astype(np.uint32)
    d = (a + np.tile(np.arange(b), a)).astype(np.uint32)
    g = orc.csr(a + b, s, d)
    deg, mu = orc.pattern_degrees(g, orc.LOOP4)
    assert mu == math.comb(a, 2) * math.comb(b, 2)
    assert deg[0] == (a - 1) * math.comb(b, 2) and deg[a] == (b - 1) * math.comb(a, 2)
    # star K_{1,m}: the centre is in C(m, x) stars, each leaf in C(m-1, x-1)
    m = 6
    g = orc.csr(m + 1, np.zeros(m, np.uint32), np.arange(1, m + 1, dtype=np.uint32))
    deg, mu = orc.pattern_degrees(g, orc.STAR, 3)
    assert mu == math.comb(m, 3) and deg[0] == math.comb(m, 3)
    assert set(deg[1:].tolist()) == {math.comb(m - 1, 2)}
    # the cycle C_4 is one loop, C_5 none; a path has no loop
    for n, want in ((4, 1), (5, 0)):
        s = np.arange(n, dtype=np.uint32)
        g = orc.csr(n, s, (s + 1) % n)
        assert orc.pattern_degrees(g, orc.LOOP4)[1] == want


def _brute_core(A, n, name, x):
    best = np.zeros(n, np.int64)
    for mask in range(1, 1 << n):
        S = [v for v in range(n) if mask >> v & 1]
        deg, _ = _brute_degrees(A, S, name, x, n)
        mn = min(deg[v] for v in S)
        for v in S:
            best[v] = max(best[v], mn)
    return best


@pytest.mark.parametrize("name,x", PATTERNS)
def test_pattern_cores_brute_force(orc, name, x):
    # core(v) = max over vertex sets S containing v of the least
    # pattern-degree inside G[S] (the largest k whose (k, Psi)-core holds v)
    for seed in range(5):
        n, s, d = gg.random_small(9, 0.35 + 0.05 * seed, seed=700 + seed)
        A = _adj_sets(n, s, d)
        g = orc.csr(n, s, d)
        core, km = orc.pattern_core_decompose(g, _code(orc, name), x)
        want = _brute_core(A, n, name, x)
        assert np.array_equal(core.astype(np.int64), want), (seed, core, want)
        assert km == int(want.max())
        levels, size, mu = orc.pattern_level_stats(g, _code(orc, name), x, core)
        for k, sz, m in zip(levels.tolist(), size.tolist(), mu.tolist()):
            S = [v for v in range(n) if core[v] >= k]
            assert sz == len(S) and m == _brute_degrees(A, S, name, x, n)[1]
            # every vertex of R_k is in >= k instances inside R_k
            dS, _ = _brute_degrees(A, S, name, x, n)
            assert all(dS[v] >= k for v in S)


def test_pattern_core_app_densest_level(orc):
    n, s, d = gg.random_small(60, 0.12, seed=808)
    g = orc.csr(n, s, d)
    for code, x in ((orc.STAR, 2), (orc.LOOP4, 0)):
        r = orc.pattern_core_app(g, code, x)
        core, km = orc.pattern_core_decompose(g, code, x)
        levels, size, mu = orc.pattern_level_stats(g, code, x, core)
        dens = [orc.density(m, z) for m, z in zip(mu, size)]
        assert orc.density(r["densest_mu"], r["densest_size"]) == max(dens)
        assert r["kmax"] == km and r["kmax_core_mu"] == int(mu[-1])


def _alive_degrees(A, alive):
    return {v: len(A[v] & alive) for v in alive}


@pytest.mark.parametrize("x", [2, 3])
def test_star_decrements_closed_form(orc, x):
    # appendix 1.2: removing v lowers a neighbour u by C(y-1, x-1) + C(z_u-1, x-1)
    # (y, z_u: alive degrees before the removal) and a 2-hop vertex w reached
    # through u by C(z_u-2, x-2) per such u; the oracle's recounts agree
    for seed in range(6):
        n, s, d = gg.random_small(12, 0.4, seed=1100 + seed)
        A = _adj_sets(n, s, d)
        g = orc.csr(n, s, d)
        before, _ = orc.pattern_degrees(g, orc.STAR, x)
        for v in range(n):
            alive = np.ones(n, np.uint8)
            alive[v] = 0
            after, _ = orc.pattern_degrees(g, orc.STAR, x, alive)
            z = _alive_degrees(A, set(range(n)))
            y = z[v]
            want = {u: 0 for u in range(n) if u != v}
            for u in A[v]:
                want[u] += math.comb(y - 1, x - 1) + math.comb(z[u] - 1, x - 1)
                for w in A[u]:
                    if w != v:
                        want[w] += math.comb(z[u] - 2, x - 2) if z[u] >= 2 else 0
            for u in want:
                assert int(before[u]) - int(after[u]) == want[u], (seed, v, u)


def test_loop_decrements_closed_form(orc):
    # appendix 2.2: group the 2-paths v - a - w by w (y_w of them); removing v
    # lowers w by C(y_w, 2) and each a of the group by y_w - 1
    for seed in range(6):
        n, s, d = gg.random_small(12, 0.45, seed=1200 + seed)
        A = _adj_sets(n, s, d)
        g = orc.csr(n, s, d)
        before, _ = orc.pattern_degrees(g, orc.LOOP4)
        for v in range(n):
            alive = np.ones(n, np.uint8)
            alive[v] = 0
            after, _ = orc.pattern_degrees(g, orc.LOOP4, 0, alive)
            want = {u: 0 for u in range(n) if u != v}
            groups = {}
            for a in A[v]:
                for w in A[a]:
                    if w != v:
                        groups.setdefault(w, []).append(a)
            for w, path_mids in groups.items():
                yw = len(path_mids)
                want[w] += math.comb(yw, 2)
                for a in path_mids:
                    want[a] += yw - 1
            for u in want:
                assert int(before[u]) - int(after[u]) == want[u], (seed, v, u)
