"""h >= 4 on graphs whose degeneracy exceeds 1024: candidate sets larger
than the bitmap tier (more than 1024 higher-ranked neighbours) are split by
their next member until they fit.  Checked against closed forms on K_1100
and element by element against the oracle on a dense bipartite graph with a
sparse sprinkle of edges inside each side (degeneracy above 1024, few enough
cliques for the oracle)."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

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


def bipartite_plus(a, inside, seed):
    """K_{a,a} on 0..a-1 / a..2a-1 plus `inside` random edges inside each side."""
    rng = np.random.default_rng(seed)
    left, right = np.meshgrid(np.arange(a), np.arange(a, 2 * a), indexing="ij")
    s = [left.ravel(), ]
    d = [right.ravel(), ]
    for off in (0, a):
        u = rng.integers(0, a, inside) + off
        v = rng.integers(0, a, inside) + off
        s.append(u)
        d.append(v)
    return 2 * a, np.concatenate(s).astype(np.uint32), np.concatenate(d).astype(np.uint32)


@pytest.mark.parametrize("h", [4, 5])
def test_k1100_closed_form(L, h):
    n = 1100
    iu = np.triu_indices(n, 1)
    with L.Graph.from_edges(n, iu[0].astype(np.uint32), iu[1].astype(np.uint32)) as g:
        deg, mu = g.clique_degrees(h)
        assert mu == comb(n, h)
        assert np.all(deg == comb(n - 1, h - 1))
        core, kmax = g.core_decompose(h)
        assert kmax == comb(n - 1, h - 1) and np.all(core == kmax)
        r = g.core_app(h, sets=False)
        assert (r["densest_mu"], r["densest_size"]) == (comb(n, h), n)


@pytest.mark.parametrize("h", [4, 5])
def test_bipartite_plus_against_oracle(L, orc, h):
    n, s, d = bipartite_plus(1100, 3000, seed=41 + h)
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        core2, rank, degen = g.degeneracy_order()
        deg, mu = g.clique_degrees(h)
        core, kmax = g.core_decompose(h)
        r = g.core_app(h)
    assert degen > 1024
    wdeg, wmu = orc.clique_degrees(og, h)
    assert mu == wmu and np.array_equal(deg, wdeg)
    wcore, wk = orc.core_decompose(og, h)
    assert kmax == wk and np.array_equal(core, wcore)
    w = orc.core_app(og, h, wcore, wk)
    assert np.array_equal(r["kmax_core"], w["kmax_core"])
    assert np.array_equal(r["densest"], w["densest"])
    assert (r["densest_mu"], r["densest_size"]) == (w["densest_mu"], w["densest_size"])


def test_peelapp_bipartite_plus_against_oracle(L, orc):
    """PeelApp (Algorithm 2) at h = 4 on a graph of degeneracy above 1024:
    its big candidate sets take the split tier; the set, its density and the
    whole removal order equal the oracle's one-at-a-time peel."""
    n, s, d = bipartite_plus(1100, 3000, seed=45)
    og = orc.csr(n, s, d)
    w = orc.peel_app(og, 4)
    with L.Graph.from_edges(n, s, d) as g:
        assert g.degeneracy_order()[2] > 1024
        r = g.peel_app(4)
    assert (r["mu"], r["size"]) == (w["mu"], w["size"])
    assert np.array_equal(np.asarray(r["order"]).astype(np.uint32), w["order"])
    assert np.array_equal(np.asarray(r["set"]).astype(np.uint32), w["set"])
