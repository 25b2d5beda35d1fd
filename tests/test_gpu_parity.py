"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Everything here is integer work, so the bar is bit-exact equality:
clique-degrees, mu, core numbers, k_max, the level statistics, the
(k_max,Psi)-core and the densest level set with its exact density.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

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


def compare_all(L, orc, n, s, d, hs, sets=True, csr=True):
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        assert g.n == n and g.m == og.m
        if csr:
            off, adj = g.csr()
            assert np.array_equal(off, og.off)
            assert np.array_equal(adj, og.adj)
        for h in hs:
            deg, mu = g.clique_degrees(h)
            wdeg, wmu = orc.clique_degrees(og, h)
            assert mu == wmu, ("mu", h)
            assert np.array_equal(deg, wdeg), ("deg", h)
            core, kmax = g.core_decompose(h)
            wcore, wk = orc.core_decompose(og, h)
            assert kmax == wk, ("kmax", h)
            assert np.array_equal(core, wcore), ("core", h)
            lk, ls, lm = g.level_stats(h)
            wk_, ws_, wm_ = orc.level_stats(og, h, wcore)
            assert np.array_equal(lk, wk_) and np.array_equal(ls, ws_) and np.array_equal(lm, wm_)
            if sets:
                r = g.core_app(h)
                w = orc.core_app(og, h, wcore, wk)
                assert r["kmax"] == w["kmax"]
                assert np.array_equal(r["kmax_core"], w["kmax_core"]), ("kmax core", h)
                assert r["kmax_core_mu"] == w["kmax_core_mu"]
                assert r["best_k"] == w["best_k"], ("best k", h)
                assert np.array_equal(r["densest"], w["densest"]), ("densest", h)
                assert (r["densest_mu"], r["densest_size"]) == (w["densest_mu"], w["densest_size"])


def test_small_random_graphs(L, orc):
    rng = np.random.default_rng(2024)
    for i in range(30):
        n = int(rng.integers(1, 70))
        p = float(rng.choice([0.05, 0.2, 0.5, 0.9]))
        n, s, d = gg.random_small(n, p, seed=300 + i)
        compare_all(L, orc, n, s, d, (2, 3, 4, 5, 6))


def test_edge_cases(L, orc):
    # n = 0
    compare_all(L, orc, 0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), (2, 3), csr=False)
    # isolated vertices only
    compare_all(L, orc, 7, np.zeros(0, np.uint32), np.zeros(0, np.uint32), (2, 3, 4))
    # one vertex with a self-loop
    compare_all(L, orc, 1, np.array([0], np.uint32), np.array([0], np.uint32), (2, 3))
    # K_60 + isolated vertices: every core value = C(59, h-1)
    s, d = np.triu_indices(60, 1)
    compare_all(L, orc, 64, s.astype(np.uint32), d.astype(np.uint32), (2, 3, 4, 5))
    # star and complete bipartite (triangle-free)
    compare_all(L, orc, 40, np.zeros(39, np.uint32), np.arange(1, 40, dtype=np.uint32), (2, 3))
    a = np.repeat(np.arange(5), 9).astype(np.uint32)
    b = (5 + np.tile(np.arange(9), 5)).astype(np.uint32)
    compare_all(L, orc, 14, a, b, (2, 3, 4))


def test_closed_form_clique(L):
    n = 45
    s, d = np.triu_indices(n, 1)
    with L.Graph.from_edges(n, s.astype(np.uint32), d.astype(np.uint32)) as g:
        for h in (2, 3, 4, 5, 6, 7, 8):
            deg, mu = g.clique_degrees(h)
            assert mu == math.comb(n, h)
            assert set(deg.tolist()) == {math.comb(n - 1, h - 1)}
            core, kmax = g.core_decompose(h)
            assert kmax == math.comb(n - 1, h - 1) and set(core.tolist()) == {kmax}


def test_large_clique_tiers(L):
    # K_1500: every out-neighbourhood above the block bitmap size (1024) goes
    # through the large h = 3 tier; one level holds every vertex
    n = 1500
    s, d = np.triu_indices(n, 1)
    with L.Graph.from_edges(n, s.astype(np.uint32), d.astype(np.uint32)) as g:
        for h in (2, 3):
            deg, mu = g.clique_degrees(h)
            assert mu == math.comb(n, h)
            assert set(deg.tolist()) == {math.comb(n - 1, h - 1)}
            core, kmax = g.core_decompose(h)
            assert kmax == math.comb(n - 1, h - 1) and set(core.tolist()) == {kmax}
            r = g.core_app(h)
            assert r["densest_size"] == n and r["densest_mu"] == math.comb(n, h)
        e = g.core_exact(2)   # (h = 3 would need a 3.4e9-arc network)
        assert e["size"] == n and e["mu"] == math.comb(n, 2)


def test_rejects_bad_input(L):
    with pytest.raises(L.DSDError) as ei:
        L.Graph.from_edges(5, np.array([0, 5], np.uint32), np.array([1, 1], np.uint32))
    assert ei.value.name == "DSD_ERR_INVALID"
    with L.Graph.from_edges(3, np.array([0], np.uint32), np.array([1], np.uint32)) as g:
        for h in (1, 9):
            with pytest.raises(L.DSDError):
                g.clique_degrees(h)


def test_device_memory_outputs(L, orc):
    import torch
    n, s, d = gg.random_small(200, 0.1, seed=77)
    og = orc.csr(n, s, d)
    st = torch.from_numpy(s.astype(np.int32)).cuda()
    dt = torch.from_numpy(d.astype(np.int32)).cuda()
    with L.Graph.from_edges(n, st, dt) as g:
        deg, mu = g.clique_degrees(3, mem="device")
        wdeg, wmu = orc.clique_degrees(og, 3)
        assert mu == wmu and np.array_equal(deg.cpu().numpy().astype(np.uint64), wdeg)
        core, kmax = g.core_decompose(3, mem="device")
        wcore, wk = orc.core_decompose(og, 3)
        assert kmax == wk and np.array_equal(core.cpu().numpy().astype(np.uint64), wcore)
        r = g.core_app(3, mem="device")
        w = orc.core_app(og, 3, wcore, wk)
        assert np.array_equal(r["kmax_core"].cpu().numpy().astype(np.uint32), w["kmax_core"])
        assert np.array_equal(r["densest"].cpu().numpy().astype(np.uint32), w["densest"])


def test_from_csr_matches_edges(L, orc):
    n, s, d = gg.random_small(150, 0.08, seed=5)
    og = orc.csr(n, s, d)
    with L.Graph.from_csr(n, og.off, og.adj) as g:
        off, adj = g.csr()
        assert np.array_equal(off, og.off) and np.array_equal(adj, og.adj)
        core, kmax = g.core_decompose(3)
        wcore, wk = orc.core_decompose(og, 3)
        assert np.array_equal(core, wcore)


def test_degeneracy_order_properties(L, orc):
    n, s, d = gg.chung_lu(20000, 100000, 2.2, 500.0, 8)
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        core2, rank, degen = g.degeneracy_order()
        wcore, wk = orc.core_decompose(og, 2)
        assert np.array_equal(core2.astype(np.uint64), wcore) and degen == wk
        assert np.array_equal(np.sort(rank), np.arange(n, dtype=np.uint32))
        # every vertex has at most core_2(v) neighbours ranked after it
        src = np.repeat(np.arange(n), np.diff(og.off).astype(np.int64))
        later = rank[og.adj] > rank[src]
        outdeg = np.bincount(src[later], minlength=n)
        assert np.all(outdeg <= core2)


@pytest.mark.parametrize("name,hs", [("er2000", (2, 3)), ("cl50k", (2, 3, 4)), ("rmat14", (3, 4, 5))])
def test_scaled_workloads(L, orc, name, hs):
    n, s, d, _ = gg.workload(name)
    compare_all(L, orc, n, s, d, hs)


@pytest.mark.parametrize("limit", [0, 1024, 3000])
def test_peel_regimes(L, orc, limit):
    """The peel's two round structures (global lists with several barriers
    per round; alive set replicated in shared memory with one barrier) and
    the switch between them give the same results."""
    L.dsd_set_peel_small_limit(limit)
    try:
        n, s, d, _ = gg.workload("cl50k")
        compare_all(L, orc, n, s, d, (2, 3, 4), csr=False)
        for i in range(4):
            n, s, d = gg.random_small(300, 0.08, seed=900 + i)
            compare_all(L, orc, n, s, d, (2, 3, 5), csr=False)
    finally:
        L.dsd_set_peel_small_limit(16384)


@pytest.mark.parametrize("tail", [0, 64, 1000, 8000, 1 << 30])
def test_peel_tail_limits(L, orc, tail):
    """The cluster tail kernel (h = 2, 3: the alive subgraph as bitmap rows in
    distributed shared memory) finishes the levels exactly as the persistent
    kernel does, whatever the hand-over size."""
    L.dsd_set_peel_tail_limit(tail)
    try:
        n, s, d, _ = gg.workload("cl50k")
        compare_all(L, orc, n, s, d, (2, 3), csr=False)
        with L.Graph.from_edges(n, s, d) as g:
            g.core_app(3)
            st = L.dsd_peel_stats(g.handle, 1)
            if tail == 0:
                assert st["tail_n"] == 0
            elif tail >= 1000:
                assert 0 < st["tail_n"] <= tail
        for i in range(4):
            n, s, d = gg.random_small(400, 0.06, seed=950 + i)
            compare_all(L, orc, n, s, d, (2, 3, 4), csr=False)
        # a dense block peeled entirely inside the tail, and an empty one
        n, s, d = gg.er(600, 0.3, seed=5)
        compare_all(L, orc, n, s, d, (2, 3), csr=False)
        compare_all(L, orc, 50, np.zeros(0, np.uint32), np.zeros(0, np.uint32), (2, 3),
                    csr=False)
    finally:
        L.dsd_set_peel_tail_limit(1 << 30)


def test_er2000_bruteforce_subsamples(L, orc):
    """Configuration 1: 16-vertex induced subsamples against brute force."""
    import bruteforce as bf
    n, s, d, _ = gg.workload("er2000")
    og = orc.csr(n, s, d)
    rng = np.random.default_rng(1)
    A_full = None
    for seed in range(1, 9):
        rng = np.random.default_rng(seed)
        # grow a connected-ish 16-vertex sample by BFS from a random vertex
        start = int(rng.integers(0, n))
        pick = [start]
        frontier = [start]
        while len(pick) < 16 and frontier:
            v = frontier.pop(0)
            for u in og.adj[og.off[v]:og.off[v + 1]].tolist():
                if u not in pick and len(pick) < 16:
                    pick.append(u)
                    frontier.append(u)
        pick = sorted(pick)
        idx = {v: i for i, v in enumerate(pick)}
        ss, dd = [], []
        for v in pick:
            for u in og.adj[og.off[v]:og.off[v + 1]].tolist():
                if u in idx and u > v:
                    ss.append(idx[v])
                    dd.append(idx[u])
        k = len(pick)
        ss = np.array(ss, np.uint32)
        dd = np.array(dd, np.uint32)
        sub = orc.csr(k, ss, dd)
        A = bf.adjacency(k, sub.off, sub.adj)
        with L.Graph.from_edges(k, ss, dd) as g:
            for h in (2, 3):
                core, _ = g.core_decompose(h)
                assert core.astype(np.int64).tolist() == bf.core_numbers(A, h).tolist()


_ITEM_CASES = {}


def _item_cases(orc):
    """Graphs for the item-path test and the oracle's core numbers (computed once)."""
    if not _ITEM_CASES:
        graphs = [gg.workload("rmat14")[:3]] + [gg.random_small(300, 0.12, seed=970 + i)
                                                 for i in range(3)]
        for gi, (n, s, d) in enumerate(graphs):
            og = orc.csr(n, s, d)
            for h in (4, 5):
                _ITEM_CASES[(gi, h)] = ((n, s, d), orc.core_decompose(og, h))
    return _ITEM_CASES


@pytest.mark.parametrize("warp_max,mid_max", [(32, 0), (4, 0), (4, 1), (2, 1 << 20), (8, 16)])
def test_peel_item_paths(L, orc, warp_max, mid_max):
    """h >= 4: the work items of the peel listed by a warp, by a group of
    warps (mid items, with the list overflowing at mid_max) or by a block
    give the oracle's core numbers whatever the thresholds."""
    cases = _item_cases(orc)
    L.dsd_set_peel_items(warp_max, mid_max)
    try:
        for (gi, h), ((n, s, d), (wcore, wk)) in cases.items():
            with L.Graph.from_edges(n, s, d) as g:
                core, kmax = g.core_decompose(h)
            assert kmax == wk, (gi, h)
            assert np.array_equal(core, wcore), (gi, h)
    finally:
        L.dsd_set_peel_items(4, 1 << 20)
