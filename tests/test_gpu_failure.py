"""Failure detection without a GPU fault: every grid-barrier wait of the
peeling kernel is bounded in time.  Withholding one block makes the others'
waits run out; the call must return DSD_ERR_TIMEOUT promptly and leave the
context usable for the next computation."""
from __future__ import annotations

import time

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


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def test_barrier_passes_when_all_blocks_arrive(L):
    L.dsd_check_barrier_timeout(-1, 2000, _stream())


@pytest.mark.parametrize("absent", [0, 7])
def test_barrier_wait_runs_out(L, orc, absent):
    t0 = time.perf_counter()
    with pytest.raises(L.DSDError) as ei:
        L.dsd_check_barrier_timeout(absent, 200, _stream())
    dt = time.perf_counter() - t0
    assert ei.value.name == "DSD_ERR_TIMEOUT"
    assert "withheld" in str(ei.value)
    assert 0.19 <= dt < 10.0
    # the context is still usable: a decomposition right after is exact
    n, s, d = gg.er(400, 0.05, seed=3)
    og = orc.csr(n, s, d)
    with L.Graph.from_edges(n, s, d) as g:
        core, kmax = g.core_decompose(3)
    wcore, wk = orc.core_decompose(og, 3)
    assert kmax == wk and np.array_equal(core, wcore)
    L.dsd_check_barrier_timeout(-1, 2000, _stream())


def test_barrier_check_rejects_bad_arguments(L):
    for args in [(0, 0), (0, 600000), (100000, 100)]:
        with pytest.raises(L.DSDError) as ei:
            L.dsd_check_barrier_timeout(args[0], args[1], _stream())
        assert ei.value.name == "DSD_ERR_INVALID"
