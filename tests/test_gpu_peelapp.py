"""PeelApp (Algorithm 2) on the GPU against the oracle's one-at-a-time
peel: the returned set, its clique count and size, and the whole removal
order, element by element (ties of the minimum clique-degree go to the
smaller id on both sides)."""
from __future__ import annotations

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


def check(L, orc, n, s, d, h, mem="host"):
    og = orc.csr(n, s, d)
    w = orc.peel_app(og, h)
    with L.Graph.from_edges(n, s, d) as g:
        r = g.peel_app(h, mem=mem)
    got_set = np.asarray(r["set"].cpu() if mem == "device" else r["set"]).astype(np.uint32)
    got_order = np.asarray(r["order"].cpu() if mem == "device" else r["order"]).astype(np.uint32)
    assert (r["mu"], r["size"]) == (w["mu"], w["size"]), (h, r["mu"], r["size"], w)
    assert np.array_equal(got_order, w["order"]), h
    assert np.array_equal(got_set, w["set"]), h
    assert r["removed"] == n - r["size"]
    return r


@pytest.mark.parametrize("h", [2, 3, 4, 5])
def test_peelapp_random(L, orc, h):
    for seed in range(6):
        n, s, d = gg.random_small(40 + 30 * seed, 0.15 + 0.05 * (seed % 3), seed=500 + seed)
        check(L, orc, n, s, d, h)


@pytest.mark.parametrize("h", [2, 3, 4])
def test_peelapp_planted_power_law(L, orc, h):
    n, s, d, _ = gg.plant(3000, *gg.chung_lu(3000, 24000, 2.1, 200.0, 17)[1:], 35, 0.7, 18)
    check(L, orc, n, s, d, h)
    check(L, orc, n, s, d, h, mem="device")


def test_peelapp_closed_forms(L, orc):
    # K_n: nothing beats the whole clique; two disjoint cliques; no edge
    k8 = np.array([(a, b) for a in range(8) for b in range(a + 1, 8)], np.uint32)
    r = check(L, orc, 8, k8[:, 0], k8[:, 1], 3)
    assert (r["mu"], r["size"]) == (56, 8)
    two = np.concatenate([k8, k8 + 8])
    extra = np.array([(a, b) for a in range(16, 22) for b in range(a + 1, 22)], np.uint32)
    both = np.concatenate([two, extra])
    check(L, orc, 22, both[:, 0], both[:, 1], 3)
    e = np.zeros(0, np.uint32)
    r = check(L, orc, 7, e, e, 3)
    assert (r["mu"], r["size"]) == (0, 7)
    r = check(L, orc, 1, e, e, 2)
    assert r["size"] == 1


def test_peelapp_cl50k(L, orc):
    n, s, d, _ = gg.workload("cl50k")
    check(L, orc, n, s, d, 3)


@pytest.mark.parametrize("shared,glob", [(0, 0), (64, 1 << 26), (600, 0), (2000, 3000)])
def test_peelapp_queue_placements(L, orc, shared, glob):
    """Every placement of the per-level bucket queues gives the oracle's
    order: no queue (a scan of the level per step), queues in global memory
    (a tiny shared budget), the buckets of the smallest counts only with the
    scan behind them, and a global budget that runs out part way."""
    L.dsd_set_peel_app_queue(shared, glob)
    try:
        n, s, d, _ = gg.plant(3000, *gg.chung_lu(3000, 24000, 2.1, 200.0, 17)[1:], 35, 0.7, 18)
        for h in (3, 4):
            check(L, orc, n, s, d, h)
        for seed in range(3):
            n, s, d = gg.random_small(120 + 40 * seed, 0.2, seed=640 + seed)
            check(L, orc, n, s, d, 3)
    finally:
        L.dsd_set_peel_app_queue(12288, 1 << 26)
