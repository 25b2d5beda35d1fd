"""GB300 (sm_103a) implementation of the data-parallel hot path of core-based
densest subgraph discovery (Fang et al., PVLDB 12(11), 2019):
h-clique clique-degrees, (k,Psi)-core decomposition and CoreApp outputs.

The compute lives in libdsd.so (CUDA, C ABI in include/dsd.h); this package
holds the ctypes binding (``_lib``), the in-tree build script (``build``) and
the seeded input generators (``graphgen``).
"""
from . import graphgen  # noqa: F401

__all__ = ["graphgen", "lib"]


def lib():
    """The ctypes binding module (loads libdsd.so; raises if it is missing)."""
    from . import _lib
    _lib.load()
    return _lib
