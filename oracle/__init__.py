"""CPU oracle (test infrastructure only).

Plain, slow, single-threaded implementations of what the GPU path computes,
written from the paper (Fang et al., PVLDB 2019): clique-degrees (Def. 3),
the (k,Psi)-core decomposition (Algorithm 3), the (k,Psi)-core by threshold
pruning (Def. 6), level statistics of the nested cores, the CoreApp
outputs (Algorithms 5 and 6; Pruning1 of Sec. 5.1), and the exact CDS by
Algorithm 1 (Exact) with its minimum cuts.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library.  The arithmetic lives in ``oracle.c`` (built with gcc by
:func:`build`); this module only marshals numpy arrays and combines the
exact integer results (densities as fractions, compared by
cross-multiplication with Python integers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.orc_build_csr.restype = ctypes.c_int64
    lib.orc_build_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _u64p, _u32p]
    lib.orc_clique_degrees.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, _u64p, _u64p]
    lib.orc_vertex_clique_degree.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                             ctypes.c_uint32, _u64p]
    lib.orc_vertex_clique_degrees.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                              _u32p, ctypes.c_uint32, _u64p]
    lib.orc_induced_clique_count.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                             _u8p, _u64p]
    lib.orc_core_decompose.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                       ctypes.c_int, _u64p, _u64p]
    lib.orc_threshold_prune.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                        ctypes.c_uint64, _u8p]
    lib.orc_level_stats.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, _u64p,
                                    _u64p, ctypes.c_uint32, _u64p, _u64p]
    lib.orc_pattern_degrees.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                        ctypes.c_int, _u8p, _u64p, _u64p]
    lib.orc_pattern_core_decompose.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                               ctypes.c_int, _u64p, _u64p]
    lib.orc_pattern_level_stats.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                            ctypes.c_int, _u64p, _u64p, ctypes.c_uint32,
                                            _u64p, _u64p]
    lib.orc_exact_cds.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, _u8p, _u64p,
                                  _u64p, _u32p]
    lib.orc_exact_cds.restype = ctypes.c_int
    lib.orc_densest_check.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint64, _u8p,
                                      ctypes.POINTER(ctypes.c_int)]
    lib.orc_densest_check.restype = ctypes.c_int
    lib.orc_peel_app.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, _u8p, _u64p,
                                 _u64p, _u32p]
    lib.orc_peel_app.restype = ctypes.c_int
    for f in ("orc_pattern_degrees", "orc_pattern_core_decompose", "orc_pattern_level_stats"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("orc_clique_degrees", "orc_vertex_clique_degree", "orc_vertex_clique_degrees",
              "orc_induced_clique_count",
              "orc_core_decompose", "orc_threshold_prune", "orc_level_stats"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle error %d" % rc)


class Graph:
    """A simple undirected graph as a sorted, symmetric CSR (original ids)."""

    def __init__(self, n, off, adj):
        self.n = int(n)
        self.off = np.ascontiguousarray(off, np.uint64)
        self.adj = np.ascontiguousarray(adj, np.uint32)

    @property
    def m(self) -> int:
        return int(self.off[-1]) // 2

    def degree(self) -> np.ndarray:
        return np.diff(self.off).astype(np.uint64)


def csr(n, src, dst) -> Graph:
    """Sec. 2 data model: symmetrise, drop self-loops and repeated pairs."""
    lib = _load()
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    m = src.size
    off = np.zeros(n + 1, np.uint64)
    adj = np.zeros(max(2 * m, 1), np.uint32)
    k = lib.orc_build_csr(n, m, _p(src, _u32p), _p(dst, _u32p), _p(off, _u64p), _p(adj, _u32p))
    if k < 0:
        raise ValueError("edge endpoint out of range" if k == -1 else "oracle error %d" % k)
    return Graph(n, off, adj[:k].copy())


def clique_degrees(g: Graph, h: int):
    """(deg[v], mu): clique-degrees (Def. 3) and the instance count (Def. 4)."""
    lib = _load()
    deg = np.zeros(max(g.n, 1), np.uint64)
    mu = np.zeros(1, np.uint64)
    _check(lib.orc_clique_degrees(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h,
                                  _p(deg, _u64p), _p(mu, _u64p)))
    return deg[:g.n], int(mu[0])


def vertex_clique_degree(g: Graph, h: int, v: int) -> int:
    lib = _load()
    out = np.zeros(1, np.uint64)
    _check(lib.orc_vertex_clique_degree(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, v,
                                        _p(out, _u64p)))
    return int(out[0])


def vertex_clique_degrees(g: Graph, h: int, vs) -> np.ndarray:
    """Def. 3 for each vertex of vs (one listing order for all)."""
    lib = _load()
    vs = np.ascontiguousarray(vs, np.uint32)
    out = np.zeros(max(vs.size, 1), np.uint64)
    _check(lib.orc_vertex_clique_degrees(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h,
                                         _p(vs, _u32p), vs.size, _p(out, _u64p)))
    return out[: vs.size]


def induced_clique_count(g: Graph, h: int, mask) -> int:
    lib = _load()
    mask = np.ascontiguousarray(np.asarray(mask, bool).astype(np.uint8))
    out = np.zeros(1, np.uint64)
    _check(lib.orc_induced_clique_count(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h,
                                        _p(mask, _u8p), _p(out, _u64p)))
    return int(out[0])


def core_decompose(g: Graph, h: int, tie_order: int = 0):
    """(core[v], kmax) by Algorithm 3."""
    lib = _load()
    core = np.zeros(max(g.n, 1), np.uint64)
    kmax = np.zeros(1, np.uint64)
    _check(lib.orc_core_decompose(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, tie_order,
                                  _p(core, _u64p), _p(kmax, _u64p)))
    return core[:g.n], int(kmax[0])


def threshold_prune(g: Graph, h: int, k: int) -> np.ndarray:
    """Boolean mask of the (k,Psi)-core R_k (Def. 6), by repeated deletion."""
    lib = _load()
    out = np.zeros(max(g.n, 1), np.uint8)
    _check(lib.orc_threshold_prune(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, int(k),
                                   _p(out, _u8p)))
    return out[:g.n].astype(bool)


def level_stats(g: Graph, h: int, core):
    """Sorted distinct levels k with |R_k| and mu(R_k) for each."""
    lib = _load()
    core = np.ascontiguousarray(core, np.uint64)
    levels = np.unique(core).astype(np.uint64)
    nl = levels.size
    size = np.zeros(max(nl, 1), np.uint64)
    mu = np.zeros(max(nl, 1), np.uint64)
    _check(lib.orc_level_stats(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h,
                               _p(core, _u64p), _p(levels, _u64p), nl,
                               _p(size, _u64p), _p(mu, _u64p)))
    return levels, size[:nl], mu[:nl]


def core_app(g: Graph, h: int, core=None, kmax=None):
    """CoreApp outputs from the decomposition (Algorithms 5/6, Pruning1).

    * kmax and the (kmax,Psi)-core {v : core(v) = kmax} (Lemma 6, IncApp);
    * the densest level set S* = argmax_k rho(R_k) over the distinct levels,
      ties to the largest k, with its exact density mu(S*)/|S*|.

    With no h-clique at all kmax = 0, and both sets are all of V (the whole
    graph is the (0,Psi)-core, Example 3).
    """
    if core is None:
        core, kmax = core_decompose(g, h)
    core = np.asarray(core, np.uint64)
    if g.n == 0:
        return dict(kmax=0, kmax_core=np.zeros(0, np.uint32), kmax_core_mu=0,
                    best_k=0, densest=np.zeros(0, np.uint32), densest_mu=0, densest_size=0)
    levels, size, mu = level_stats(g, h, core)
    best = 0
    for j in range(1, levels.size):
        # rho_j >= rho_best, ties to the larger k (later j)
        if int(mu[j]) * int(size[best]) >= int(mu[best]) * int(size[j]):
            best = j
    km = int(levels[-1])
    kcore = np.nonzero(core == np.uint64(km))[0].astype(np.uint32)
    dens = np.nonzero(core >= levels[best])[0].astype(np.uint32)
    return dict(kmax=km, kmax_core=kcore, kmax_core_mu=int(mu[-1]),
                best_k=int(levels[best]), densest=dens,
                densest_mu=int(mu[best]), densest_size=int(size[best]))


def density(mu: int, size: int) -> Fraction:
    return Fraction(int(mu), int(size)) if size else Fraction(0)


def exact_cds(g: Graph, h: int):
    """The CDS by Algorithm 1 (Exact): rho_opt and the largest densest set.

    Returns dict(cds = sorted vertex ids of the union of all maximum-density
    sets, mu = its h-clique count, size = its size, steps = binary-search
    iterations); rho_opt = mu / size.  With no h-clique the answer is V with
    density 0.
    """
    lib = _load()
    mark = np.zeros(max(g.n, 1), np.uint8)
    mu = np.zeros(1, np.uint64)
    size = np.zeros(1, np.uint64)
    steps = np.zeros(1, np.uint32)
    _check(lib.orc_exact_cds(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, _p(mark, _u8p),
                             _p(mu, _u64p), _p(size, _u64p), _p(steps, _u32p)))
    cds = np.flatnonzero(mark[:g.n]).astype(np.uint32)
    return dict(cds=cds, mu=int(mu[0]), size=int(size[0]), steps=int(steps[0]))


def peel_app(g: Graph, h: int):
    """Algorithm 2 (PeelApp): the densest of G and its residuals under
    one-at-a-time removal of a minimum clique-degree vertex (ties: smaller
    id).  Returns dict(set = sorted ids, mu, size, order = the removal
    order)."""
    lib = _load()
    mark = np.zeros(max(g.n, 1), np.uint8)
    mu = np.zeros(1, np.uint64)
    size = np.zeros(1, np.uint64)
    order = np.zeros(max(g.n, 1), np.uint32)
    _check(lib.orc_peel_app(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, _p(mark, _u8p),
                            _p(mu, _u64p), _p(size, _u64p), _p(order, _u32p)))
    return dict(set=np.flatnonzero(mark[:g.n]).astype(np.uint32), mu=int(mu[0]),
                size=int(size[0]), order=order[:g.n])


def densest_check(g: Graph, h: int, p: int, q: int):
    """One minimum cut of Algorithm 1's network at alpha = p/q.

    Returns (beats, largest_source_side): beats is True when some vertex set
    has density above p/q; at p/q = rho_opt it is False and the set is the
    largest densest set (sorted ids).
    """
    lib = _load()
    mark = np.zeros(max(g.n, 1), np.uint8)
    beats = ctypes.c_int(0)
    _check(lib.orc_densest_check(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), h, int(p), int(q),
                                 _p(mark, _u8p), ctypes.byref(beats)))
    return bool(beats.value), np.flatnonzero(mark[:g.n]).astype(np.uint32)


# ------------------------------------------------------------ patterns (Sec. 6)

STAR = 1     # x-star: a centre and x of its neighbours
LOOP4 = 2    # the 4-vertex loop (4-cycle)


def pattern_size(pattern: int, x: int) -> int:
    return x + 1 if pattern == STAR else 4


def pattern_degrees(g: Graph, pattern: int, x: int = 0, alive=None):
    """Pattern-degrees (Sec. 6) of every vertex and mu; alive: optional mask."""
    lib = _load()
    deg = np.zeros(max(g.n, 1), np.uint64)
    mu = np.zeros(1, np.uint64)
    m = None
    if alive is not None:
        m = np.ascontiguousarray(alive, np.uint8)
    _check(lib.orc_pattern_degrees(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), pattern, x,
                                   _p(m, _u8p) if m is not None else None, _p(deg, _u64p),
                                   _p(mu, _u64p)))
    return deg[:g.n], int(mu[0])


def pattern_core_decompose(g: Graph, pattern: int, x: int = 0):
    """Algorithm 3 extended to a pattern: (core numbers, k_max)."""
    lib = _load()
    core = np.zeros(max(g.n, 1), np.uint64)
    km = np.zeros(1, np.uint64)
    _check(lib.orc_pattern_core_decompose(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), pattern, x,
                                          _p(core, _u64p), _p(km, _u64p)))
    return core[:g.n], int(km[0])


def pattern_level_stats(g: Graph, pattern: int, x: int, core):
    """(levels k, |R_k|, mu(R_k)) for the distinct core values, ascending."""
    lib = _load()
    core = np.ascontiguousarray(core, np.uint64)
    levels = np.unique(core) if g.n else np.zeros(0, np.uint64)
    levels = np.ascontiguousarray(levels, np.uint64)
    nl = levels.size
    size = np.zeros(max(nl, 1), np.uint64)
    mu = np.zeros(max(nl, 1), np.uint64)
    _check(lib.orc_pattern_level_stats(g.n, _p(g.off, _u64p), _p(g.adj, _u32p), pattern, x,
                                       _p(core, _u64p), _p(levels, _u64p), nl, _p(size, _u64p),
                                       _p(mu, _u64p)))
    return levels, size[:nl], mu[:nl]


def pattern_core_app(g: Graph, pattern: int, x: int = 0):
    """k_max, the (k_max, Psi)-core, and the densest level set (ties to the
    larger k) with its exact pattern-density, for a pattern (Sec. 6)."""
    core, km = pattern_core_decompose(g, pattern, x)
    levels, size, mu = pattern_level_stats(g, pattern, x, core)
    if g.n == 0:
        return dict(kmax=0, kmax_core=np.zeros(0, np.uint32), kmax_core_mu=0, best_k=0,
                    densest=np.zeros(0, np.uint32), densest_mu=0, densest_size=0)
    best = 0
    for j in range(1, len(levels)):
        if density(mu[j], size[j]) >= density(mu[best], size[best]):
            best = j
    bk = int(levels[best])
    return dict(kmax=km, kmax_core=np.flatnonzero(core >= km).astype(np.uint32),
                kmax_core_mu=int(mu[-1]), best_k=bk,
                densest=np.flatnonzero(core >= bk).astype(np.uint32),
                densest_mu=int(mu[best]), densest_size=int(size[best]))

