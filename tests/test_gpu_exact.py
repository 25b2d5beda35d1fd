"""GPU parity of CoreExact (dsd_core_exact) against the oracle's Algorithm 1.

The answer is unique: rho_opt as an exact fraction and the largest densest
vertex set (the union of all sets of density rho_opt).  Both are compared
exactly.  Larger graphs use the oracle on the (ceil(rho'),Psi)-core only,
rho' being the oracle's own densest level: every densest set lies in that
core (each of its vertices is in >= rho_opt of its cliques, Sec. 4.3), so the
oracle's answer there is its answer on the whole graph.
"""
from __future__ import annotations

import math
from fractions import Fraction

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


def _check(r, w, ctx=""):
    assert (r["mu"], r["size"]) == (w["mu"], w["size"]), ctx
    assert np.array_equal(np.asarray(r["cds"], np.uint32), w["cds"]), ctx


def _oracle_on_core(orc, og, h):
    """The oracle's exact answer via its own (ceil(rho'),Psi)-core."""
    core, kmax = orc.core_decompose(og, h)
    app = orc.core_app(og, h, core, kmax)
    if app["densest_mu"] == 0:
        return orc.exact_cds(og, h)
    k1 = math.ceil(Fraction(app["densest_mu"], app["densest_size"]))
    keep = np.flatnonzero(core >= k1).astype(np.uint32)
    mask = np.zeros(og.n, bool)
    mask[keep] = True
    src = np.repeat(np.arange(og.n, dtype=np.uint32), np.diff(og.off).astype(np.int64))
    sel = mask[src] & mask[og.adj] & (src < og.adj)
    remap = np.full(og.n, 0, np.uint32)
    remap[keep] = np.arange(keep.size, dtype=np.uint32)
    sub = orc.csr(int(keep.size), remap[src[sel]], remap[og.adj[sel]])
    w = orc.exact_cds(sub, h)
    return dict(mu=w["mu"], size=w["size"], cds=keep[w["cds"]])


@pytest.mark.parametrize("h", [2, 3, 4, 5])
def test_exact_small(L, orc, h):
    rng = np.random.default_rng(100 + h)
    for i in range(10):
        n = int(rng.integers(6, 48))
        p = float(rng.choice([0.15, 0.3, 0.5, 0.8]))
        n, s, d = gg.random_small(n, p, seed=8000 + 17 * h + i)
        og = orc.csr(n, s, d)
        with L.Graph.from_edges(n, s, d) as g:
            r = g.core_exact(h)
        _check(r, orc.exact_cds(og, h), (h, i))


@pytest.mark.parametrize("h", [2, 3, 4])
def test_exact_planted(L, orc, h):
    for seed in range(3):
        n, s, d = gg.er(2000, 0.004, 8100 + seed)
        n, s, d, _ = gg.plant(n, s, d, 40 + 10 * seed, 0.6, 8200 + seed)
        n, s, d, _ = gg.plant(n, s, d, 25, 0.9, 8300 + seed)
        og = orc.csr(n, s, d)
        with L.Graph.from_edges(n, s, d) as g:
            r = g.core_exact(h)
            app = g.core_app(h, sets=False)
        _check(r, orc.exact_cds(og, h), (h, seed))
        # the search started from the best of Pruning1/Pruning2 and ended above it
        lower = Fraction(r["lower_mu"], r["lower_size"])
        assert lower >= Fraction(app["densest_mu"], app["densest_size"])
        assert Fraction(r["mu"], r["size"]) >= lower
        assert r["k2"] >= r["k1"] >= 1 and r["cuts"] >= 1


def test_exact_equal_components(L, orc):
    # two vertex-disjoint K_12 in a sparse background: both are returned
    n, s, d = gg.er(3000, 0.001, 8400)
    rng = np.random.default_rng(8401)
    verts = rng.choice(n, size=24, replace=False).astype(np.uint32)
    extra = [(verts[a], verts[b]) for blk in (range(0, 12), range(12, 24))
             for a in blk for b in blk if a < b]
    s = np.concatenate([s, np.array([e[0] for e in extra], np.uint32)])
    d = np.concatenate([d, np.array([e[1] for e in extra], np.uint32)])
    og = orc.csr(n, s, d)
    for h in (3, 4):
        with L.Graph.from_edges(n, s, d) as g:
            r = g.core_exact(h)
        w = orc.exact_cds(og, h)
        _check(r, w, h)
        assert set(verts.tolist()) <= set(r["cds"].tolist())


def test_exact_degenerate(L, orc):
    # no triangle (bipartite): every set has density 0, the answer is V
    a, b = 7, 9
    s = np.repeat(np.arange(a), b).astype(np.uint32)
    d = (a + np.tile(np.arange(b), a)).astype(np.uint32)
    with L.Graph.from_edges(a + b, s, d) as g:
        r = g.core_exact(3)
        assert r["mu"] == 0 and r["size"] == a + b
        assert r["cds"].tolist() == list(range(a + b))
        r2 = g.core_exact(2)
    _check(r2, orc.exact_cds(orc.csr(a + b, s, d), 2))
    # edgeless and empty graphs
    with L.Graph.from_edges(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
        r = g.core_exact(2)
        assert r["mu"] == 0 and r["cds"].tolist() == [0, 1, 2, 3, 4]
    with L.Graph.from_edges(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
        r = g.core_exact(3)
        assert r["mu"] == 0 and r["size"] == 0
    # a single clique: the whole clique
    k = 9
    iu, ju = np.triu_indices(k, 1)
    with L.Graph.from_edges(k, iu.astype(np.uint32), ju.astype(np.uint32)) as g:
        for h in (2, 3, 4, 6):
            r = g.core_exact(h)
            assert r["size"] == k and r["mu"] == math.comb(k, h)


def test_exact_device_output_and_repeat(L, orc):
    import torch
    n, s, d = gg.er(1500, 0.006, 8500)
    n, s, d, _ = gg.plant(n, s, d, 30, 0.7, 8501)
    with L.Graph.from_edges(n, s, d) as g:
        r1 = g.core_exact(3)
        r2 = g.core_exact(3, mem="device")
        r3 = g.core_exact(3)
    assert isinstance(r2["cds"], torch.Tensor)
    assert np.array_equal(r2["cds"].cpu().numpy().astype(np.uint32), r1["cds"])
    _check(r1, r3)
    _check(r1, orc.exact_cds(orc.csr(n, s, d), 3))


@pytest.mark.parametrize("h", [2, 3, 4])
def test_exact_chung_lu_50k(L, orc, h):
    n, s, d, _ = gg.workload("cl50k")
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        r = g.core_exact(h)
    _check(r, _oracle_on_core(orc, og, h), h)


def test_exact_many_components(L, orc):
    # 40 disjoint planted blocks of 8..20 vertices in a sparse background; the
    # densest blocks tie in pairs (equal sizes, both complete)
    rng = np.random.default_rng(8600)
    n, s, d = gg.er(6000, 0.0004, 8601)
    verts = rng.permutation(n).astype(np.uint32)
    at, src, dst = 0, [s], [d]
    for b in range(40):
        k = 8 + (b % 13)
        blk = verts[at:at + k]
        at += k
        iu, ju = np.triu_indices(k, 1)
        keep = (np.ones(iu.size, bool) if k >= 19 else rng.random(iu.size) < 0.8)
        src.append(blk[iu[keep]])
        dst.append(blk[ju[keep]])
    s = np.concatenate(src).astype(np.uint32)
    d = np.concatenate(dst).astype(np.uint32)
    og = orc.csr(n, s, d)
    for h in (2, 3, 4):
        with L.Graph.from_edges(n, s, d) as g:
            r = g.core_exact(h)
        _check(r, orc.exact_cds(og, h), h)
        assert r["components"] >= 1


@pytest.mark.parametrize("h", [6, 7, 8])
def test_exact_large_h(L, orc, h):
    for seed in range(3):
        n, s, d = gg.er(300, 0.03, 8700 + seed)
        n, s, d, _ = gg.plant(n, s, d, 16 + seed, 0.85, 8800 + seed)
        og = orc.csr(n, s, d)
        with L.Graph.from_edges(n, s, d) as g:
            r = g.core_exact(h)
        _check(r, orc.exact_cds(og, h), (h, seed))


def test_exact_wait_limit(L):
    # the min cut checks the wait limit between its rounds: a 1 ms limit on a
    # cut of ~50 ms ends it with DSD_ERR_TIMEOUT, and the handle and the
    # context stay usable
    n, s, d, _ = gg.workload("rmat14")
    with L.Graph.from_edges(n, s, d) as g:
        ref = g.core_exact(4)
        L.dsd_set_wait_limit_ms(1)
        try:
            with pytest.raises(L.DSDError) as ei:
                g.core_exact(4)
            assert ei.value.name == "DSD_ERR_TIMEOUT"
        finally:
            L.dsd_set_wait_limit_ms(20000)
        again = g.core_exact(4)
    _check(again, ref)
