"""Checked mode of the 64-bit counters: wrap-around turns into
DSD_ERR_OVERFLOW.  A graph whose clique counts reach 2^64 cannot be listed,
so the checked addition itself is exercised on values at the edge of the
range through dsd_checked_add_selftest (the same device routine the counting
kernels use), and the checked counting path must give the unchecked results
on real graphs."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1906_00341_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

U64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_00341_gb300 import build as b
    b.build()
    from paper_1906_00341_gb300 import _lib
    _lib.load()
    return _lib


def test_checked_add_near_the_top(L):
    start = U64 - 10
    assert L.dsd_checked_add_selftest(start, [3, 4, 3]) == (U64, False)
    assert L.dsd_checked_add_selftest(start, [3, 4, 4]) == (0, True)
    assert L.dsd_checked_add_selftest(start, [11]) == (0, True)
    assert L.dsd_checked_add_selftest(0, [U64]) == (U64, False)
    assert L.dsd_checked_add_selftest(1, [U64]) == (0, True)
    assert L.dsd_checked_add_selftest(5, []) == (5, False)


@pytest.mark.parametrize("h", [3, 4, 5])
def test_checked_counts_equal_unchecked(L, orc, h):
    n, s, d, _ = gg.plant(3000, *gg.chung_lu(3000, 30000, 2.1, 200.0, 4)[1:], 40, 0.7, 6)
    with L.Graph.from_edges(n, s, d) as g:
        deg0, mu0 = g.clique_degrees(h)
        L.dsd_set_checked(True)
        try:
            deg1, mu1 = g.clique_degrees(h)
            r1 = g.core_app(h, sets=False)
        finally:
            L.dsd_set_checked(False)
        r0 = g.core_app(h, sets=False)
    assert mu0 == mu1 and np.array_equal(deg0, deg1)
    assert r0 == r1
    wdeg, wmu = orc.clique_degrees(orc.csr(n, s, d), h)
    assert mu1 == wmu and np.array_equal(deg1, wdeg)
