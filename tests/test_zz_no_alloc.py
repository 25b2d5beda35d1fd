"""The allocation-free triangle clique-degree entry point, through the C ABI.

It serves callers that cannot allocate device memory (a host framework
whose allocator already holds the GPU's memory, a serving path that may not
allocate mid-request).  Its results must equal those of dsd_clique_degrees
with h = 3, on two calls in a row (the second call reuses the shared scratch
array left behind by the first).  The file name makes pytest collect it
last.
"""
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


@pytest.mark.parametrize("graph", ["planted_chung_lu", "random_small"])
def test_noalloc_matches_clique_degrees(L, graph):
    import torch
    if graph == "planted_chung_lu":
        # hubs at low ids give rows with more than 32 higher-id neighbours
        n, s, d, _ = gg.plant(40000, *gg.chung_lu(40000, 300000, 2.1, 900.0, 31)[1:], 40, 0.6, 32)
    else:
        n, s, d = gg.random_small(500, 0.05, seed=33)
    with L.Graph.from_edges(n, s, d) as g:
        want_deg, want_mu = g.clique_degrees(3)           # existing entry point
        off, adj = g.csr(mem="device")
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            deg = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            mu = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            L.dsd_triangle_degrees_noalloc(n, off.data_ptr(), adj.data_ptr(), deg.data_ptr(),
                                           mu.data_ptr(), stream)
            torch.cuda.synchronize()
            got = deg.cpu().numpy().astype(np.uint64)
            assert int(mu.item()) == want_mu, ("mu", call)
            assert np.array_equal(got, want_deg), ("deg", call)


def test_noalloc_edgeless_graph(L):
    """Vertices but no edges: a null adj is accepted and every count is 0."""
    import torch
    n = 1000
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        deg = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        mu = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        L.dsd_triangle_degrees_noalloc(n, off.data_ptr(), 0, deg.data_ptr(), mu.data_ptr(),
                                       stream)
        torch.cuda.synchronize()
        assert int(mu.item()) == 0 and int(deg.abs().sum().item()) == 0, call


def test_noalloc_rejects_too_many_vertices(L):
    with pytest.raises(L.DSDError) as ei:
        L.dsd_triangle_degrees_noalloc(1 << 21, 1, 1, 1, 1, 0)
    assert ei.value.name == "DSD_ERR_UNSUPPORTED"
    assert "at most" in str(ei.value)
