"""Batched executor: every graph of a mixed batch (uneven sizes, h in 2..4)
run by the persistent launch must give exactly what the single-graph path
gives (and, for a sample, what the oracle gives)."""
from __future__ import annotations

import os

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


def single(L, n, s, d, h):
    with L.Graph.from_edges(n, s, d) as g:
        r = g.core_app(h, sets=False)
        core, kmax = g.core_decompose(h)
    return r, core


def check_batch(L, graphs, orc=None, oracle_every=0):
    b = L.Batch(graphs, want_cores=True)
    b.run()
    res = b.results()
    for i, ((n, s, d, h), r) in enumerate(zip(graphs, res)):
        assert r["status"] == 0, (i, r["status"])
        want, wcore = single(L, n, s, d, h)
        for key in ("kmax", "kmax_core_size", "kmax_core_mu", "best_k", "densest_size",
                    "densest_mu", "nlevels"):
            assert r[key] == want[key], (i, n, h, key, r[key], want[key])
        assert np.array_equal(r["core"], wcore), (i, n, h)
        if orc is not None and oracle_every and i % oracle_every == 0:
            og = orc.csr(n, s, d)
            ocore, ok = orc.core_decompose(og, h)
            assert np.array_equal(r["core"], ocore) and r["kmax"] == ok
    b.close()
    return res


def test_batch_mixed_small(L, orc):
    graphs = gg.batch(48, nmax=3000, nmedian=400.0)
    check_batch(L, graphs, orc, oracle_every=4)


def test_batch_edge_cases(L):
    e = np.zeros(0, np.uint32)
    graphs = [
        (1, e, e, 2),
        (5, e, e, 3),                                                   # no edges
        (3, np.array([0, 1, 1], np.uint32), np.array([0, 1, 2], np.uint32), 2),  # loops
        (4, np.array([0, 0, 0, 1, 1, 2], np.uint32), np.array([1, 2, 3, 2, 3, 3], np.uint32), 4),
        (60, *np.triu_indices(60, 1), 3),                             # K_60
    ]
    graphs = [(n, np.asarray(s, np.uint32), np.asarray(d, np.uint32), h) for n, s, d, h in graphs]
    check_batch(L, graphs)


def test_batch_rejects_and_flags(L):
    with pytest.raises(L.DSDError) as ei:
        L.Batch([(70000, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3)])
    assert ei.value.name == "DSD_ERR_UNSUPPORTED"
    # an endpoint out of range marks that graph invalid, the others still run
    good = gg.batch_graph(1, nmax=500, nmedian=200.0)
    bad = (10, np.array([0, 11], np.uint32), np.array([1, 2], np.uint32), 3)
    b = L.Batch([good, bad])
    b.run()
    res = b.results()
    assert res[0]["status"] == 0 and res[1]["status"] == 1
    b.close()


def test_batch_autotune_cache(L, tmp_path):
    graphs = gg.batch(24, nmax=2000, nmedian=300.0)
    cache = str(tmp_path / "tune.txt")
    b1 = L.Batch(graphs, want_cores=False, autotune_cache=cache)
    t1 = b1.info()
    b1.close()
    assert os.path.exists(cache) and open(cache).read().count("|") == 1
    b2 = L.Batch(graphs, want_cores=False, autotune_cache=cache)
    t2 = b2.info()
    assert t1[:3] == t2[:3]
    # replays of the captured graph give the same answers
    b2.run()
    r1 = b2.results()
    b2.run()
    r2 = b2.results()
    assert r1 == r2
    b2.close()


def test_batch_run_over_handles(L, orc):
    """dsd_batch_run on existing graph handles: graphs within the batch
    kernel's limits run in one launch, the others (n > 65535, h > 4) through
    the single-graph path inside the same call; every result and core array
    equals dsd_core_app / dsd_core_decompose on that handle, and a sample
    equals the oracle."""
    graphs = gg.batch(20, nmax=3000, nmedian=400.0)
    big = gg.chung_lu(70000, 200000, 2.3, 300.0, 5)
    graphs.append((big[0], big[1], big[2], 3))          # beyond the batch kernel's n
    n5, s5, d5 = gg.random_small(60, 0.5, seed=9)
    graphs.append((n5, s5, d5, 5))                      # beyond its h
    handles = [L.Graph.from_edges(n, s, d) for n, s, d, _ in graphs]
    try:
        hs = [h for _, _, _, h in graphs]
        res = L.dsd_batch_run(handles, hs, want_cores=True)
        for i, ((n, s, d, h), g, r) in enumerate(zip(graphs, handles, res)):
            want = g.core_app(h, sets=False)
            core, kmax = g.core_decompose(h)
            for key in ("kmax", "kmax_core_size", "kmax_core_mu", "best_k", "densest_size",
                        "densest_mu", "nlevels"):
                assert r[key] == want[key], (i, key)
            assert np.array_equal(r["core"], core), i
            if i % 5 == 0 or i >= len(graphs) - 2:
                ocore, ok = orc.core_decompose(orc.csr(n, s, d), h)
                assert np.array_equal(r["core"], ocore) and r["kmax"] == ok, i
        # no core arrays wanted, empty call
        res2 = L.dsd_batch_run(handles[:3], hs[:3])
        assert [x["kmax"] for x in res2] == [x["kmax"] for x in res[:3]]
        assert L.dsd_batch_run([], []) == []
    finally:
        for g in handles:
            g.close()


def test_batch_every_tuned_shape_agrees(L, orc):
    """Every shape of the tuner's search space (threads x CTAs per SM x lanes
    per row scan) gives the same results, equal to the single-graph path."""
    graphs = gg.batch(48, nmax=3000, nmedian=400.0)
    b = L.Batch(graphs, want_cores=True)
    ref = None
    for threads, cps in ((256, 1), (256, 2), (512, 1), (512, 2), (1024, 1)):
        for lanes in (32, 16, 8):
            try:
                b.set_shape(threads, cps, lanes)
            except L.DSDError as e:
                assert e.name == "DSD_ERR_UNSUPPORTED"    # does not fit on an SM
                continue
            assert b.info()[:3] == (threads, cps, lanes)
            b.run()
            res = b.results()
            key = [(r["kmax"], r["best_k"], r["densest_mu"], r["densest_size"], r["nlevels"],
                    r["core"].tobytes()) for r in res]
            if ref is None:
                ref = key
                for (n, s, d, h), r in zip(graphs, res):
                    want, wcore = single(L, n, s, d, h)
                    assert r["kmax"] == want["kmax"] and np.array_equal(r["core"], wcore)
            assert key == ref, (threads, cps, lanes)
    assert ref is not None
    b.close()


def test_batch_wide_h4_graph_falls_back(L, orc):
    """An h = 4 graph with more than 512 higher-ranked neighbours at a vertex
    (a clique of 600) is answered inside the batch by the single-graph path;
    the others by the batch kernel."""
    k = 600
    iu = np.triu_indices(k, 1)
    wide = (k, iu[0].astype(np.uint32), iu[1].astype(np.uint32), 4)
    graphs = gg.batch(6, nmax=2000, nmedian=300.0) + [wide]
    b = L.Batch(graphs, want_cores=True)
    b.run()
    res = b.results()
    for (n, s, d, h), r in zip(graphs, res):
        assert r["status"] == 0
        want, wcore = single(L, n, s, d, h)
        assert r["kmax"] == want["kmax"] and np.array_equal(r["core"], wcore)
    from math import comb
    assert res[-1]["kmax"] == comb(k - 1, 3) and res[-1]["densest_mu"] == comb(k, 4)
    b.run()
    again = b.results()
    for x, y in zip(again, res):
        assert x["kmax"] == y["kmax"] and np.array_equal(x["core"], y["core"])
    b.close()
