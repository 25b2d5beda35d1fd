"""GPU parity of the pattern densities (Sec. 6: x-star and 4-loop
pattern-degrees, (k,Psi)-core numbers, level records, CoreApp outputs)
against the pattern oracle, bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1906_00341_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

PATTERNS = [("star", 2), ("star", 3), ("star", 5), ("loop", 0)]


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_00341_gb300 import build as b
    b.build()
    from paper_1906_00341_gb300 import _lib
    _lib.load()
    return _lib


def _codes(L, orc, name):
    return (L.DSD_PATTERN_STAR, orc.STAR) if name == "star" else (L.DSD_PATTERN_LOOP4, orc.LOOP4)


def _compare(L, orc, n, s, d, name, x, ctx):
    gp, op = _codes(L, orc, name)
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        deg, mu = g.pattern_degrees(gp, x)
        core, km, lk, ls, lm = g.pattern_core_decompose(gp, x)
        app = g.pattern_core_app(gp, x)
    wdeg, wmu = orc.pattern_degrees(og, op, x)
    assert mu == wmu and np.array_equal(deg, wdeg), ("degrees", ctx)
    wcore, wkm = orc.pattern_core_decompose(og, op, x)
    assert km == wkm and np.array_equal(core, wcore), ("cores", ctx)
    wlk, wls, wlm = orc.pattern_level_stats(og, op, x, wcore)
    assert np.array_equal(lk, wlk) and np.array_equal(ls, wls) and np.array_equal(lm, wlm), \
        ("levels", ctx)
    w = orc.pattern_core_app(og, op, x)
    assert app["kmax"] == w["kmax"] and app["best_k"] == w["best_k"], ctx
    assert np.array_equal(app["kmax_core"], w["kmax_core"]), ctx
    assert np.array_equal(app["densest"], w["densest"]), ctx
    assert (app["densest_mu"], app["densest_size"]) == (w["densest_mu"], w["densest_size"]), ctx
    assert app["kmax_core_mu"] == w["kmax_core_mu"], ctx


@pytest.mark.parametrize("name,x", PATTERNS)
def test_pattern_small(L, orc, name, x):
    rng = np.random.default_rng(9000 + x)
    for i in range(8):
        n = int(rng.integers(2, 40))
        n, s, d = gg.random_small(n, float(rng.choice([0.1, 0.3, 0.6])), seed=9100 + 7 * x + i)
        _compare(L, orc, n, s, d, name, x, (name, x, i))


@pytest.mark.parametrize("name,x", PATTERNS)
def test_pattern_planted(L, orc, name, x):
    n, s, d = gg.er(1500, 0.004, 9200 + x)
    n, s, d, _ = gg.plant(n, s, d, 30, 0.5, 9300 + x)
    _compare(L, orc, n, s, d, name, x, (name, x))


def test_pattern_degenerate_and_device(L, orc):
    import torch
    # edgeless, empty, and device-memory degrees
    with L.Graph.from_edges(4, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
        deg, mu = g.pattern_degrees(L.DSD_PATTERN_LOOP4)
        assert mu == 0 and deg.tolist() == [0, 0, 0, 0]
        app = g.pattern_core_app(L.DSD_PATTERN_STAR, 2)
        assert app["kmax"] == 0 and app["densest"].tolist() == [0, 1, 2, 3]
    with L.Graph.from_edges(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
        app = g.pattern_core_app(L.DSD_PATTERN_STAR, 3)
        assert app["kmax"] == 0 and app["densest_size"] == 0
    n, s, d = gg.er(500, 0.02, 9400)
    with L.Graph.from_edges(n, s, d) as g:
        dh, mh = g.pattern_degrees(L.DSD_PATTERN_STAR, 3)
        dd, md = g.pattern_degrees(L.DSD_PATTERN_STAR, 3, mem="device")
        assert isinstance(dd, torch.Tensor) and md == mh
        assert np.array_equal(dd.cpu().numpy().astype(np.uint64), dh)
        with pytest.raises(L.DSDError):
            g.pattern_degrees(L.DSD_PATTERN_STAR, 1)
        with pytest.raises(L.DSDError):
            g.pattern_degrees(7, 2)


@pytest.mark.parametrize("name,x", [("star", 2), ("star", 3), ("loop", 0)])
def test_pattern_power_law(L, orc, name, x):
    # hubs: a frontier vertex next to a hub changes the counts of the hub's
    # whole neighbourhood; many levels with several vertices leaving at once
    n, s, d = gg.chung_lu(2000, 16000, 2.1, 200.0, 9501)
    n, s, d, _ = gg.plant(n, s, d, 30, 0.5, 9502)
    _compare(L, orc, n, s, d, name, x, (name, x, "power law"))
