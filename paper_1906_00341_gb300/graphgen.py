"""Seeded synthetic graph generators.

This module only draws random edge lists; it holds none of the method's
arithmetic (no clique listing, no peeling, no densities).  Both the CPU
oracle and the CUDA path read the edge lists it returns, so that the two
sides see byte-identical inputs.

Every generator returns ``(n, src, dst)`` with ``src``/``dst`` as ``uint32``
numpy arrays.  The lists may contain self-loops and duplicate pairs in either
orientation (R-MAT and Chung-Lu draws produce them); the graph model of the
paper (Sec. 2, "Data model": undirected, unweighted, simple) is obtained by
the CSR builders on either side, which symmetrise and drop loops/duplicates.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``).

Workload shapes (the paper's real datasets are not available; these stand in
for them, Sec. 7.1 "Datasets"):

* ``er``         -- Erdos-Renyi G(n, p), like the paper's ER synthetic graph.
* ``chung_lu``   -- power-law expected-degree graph (exponent beta, capped
                    maximum expected degree), for the paper's power-law graphs.
* ``rmat``       -- recursive-matrix graph (Graph500 style), vertex labels
                    permuted, like the paper's R-MAT synthetic graph.
* ``plant``      -- adds a dense G(k, p) block on k random vertices, the
                    near-clique shape of the densest subgraphs found on real
                    graphs.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "er", "chung_lu", "rmat", "plant", "concat", "random_small",
    "workload", "WORKLOADS",
]


def _pairs_from_linear(idx: np.ndarray):
    """Map linear indices over {(u, v): u < v} (ordered by v, then u) to pairs."""
    idx = idx.astype(np.float64)
    v = np.floor((1.0 + np.sqrt(1.0 + 8.0 * idx)) / 2.0).astype(np.int64)
    idx_i = idx.astype(np.int64)
    # repair floating-point rounding at the row boundaries
    base = v * (v - 1) // 2
    too_big = base > idx_i
    v[too_big] -= 1
    base = v * (v - 1) // 2
    too_small = idx_i - base >= v
    v[too_small] += 1
    base = v * (v - 1) // 2
    u = idx_i - base
    return u.astype(np.uint32), v.astype(np.uint32)


def er(n: int, p: float, seed: int):
    """G(n, p) by geometric skipping over the n(n-1)/2 vertex pairs
    (Batagelj and Brandes, 2005).  No loops, no duplicates."""
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    if n < 2 or p <= 0.0:
        e = np.zeros(0, np.uint32)
        return n, e, e.copy()
    if p >= 1.0:
        idx = np.arange(npairs, dtype=np.int64)
    else:
        chunks = []
        pos = -1
        expect = int(npairs * p + 10 * math.sqrt(npairs * p + 1) + 16)
        while True:
            gaps = rng.geometric(p, size=expect)
            pos_arr = pos + np.cumsum(gaps, dtype=np.int64)
            keep = pos_arr[pos_arr < npairs]
            chunks.append(keep)
            if keep.size < pos_arr.size:
                break
            pos = int(pos_arr[-1])
        idx = np.concatenate(chunks) if chunks else np.zeros(0, np.int64)
    u, v = _pairs_from_linear(idx)
    return n, u, v


def chung_lu(n: int, m_draws: int, beta: float, wmax: float, seed: int,
             wsum: float | None = None):
    """Chung-Lu expected-degree graph.

    Weights w_i = c * (i + i0) ** (-1 / (beta - 1)), i = 0..n-1, with i0 and
    c chosen so that max w = ``wmax`` and sum w = ``wsum`` (default 2 *
    ``m_draws``).  ``m_draws`` endpoint pairs are drawn, each endpoint with
    probability proportional to w; loops and repeated pairs are left for the
    CSR builder to drop, so the realised edge count is a little below
    ``m_draws``.
    """
    rng = np.random.default_rng(seed)
    if wsum is None:
        wsum = 2.0 * m_draws
    gam = 1.0 / (beta - 1.0)
    i = np.arange(n, dtype=np.float64)

    def total(i0):
        w = (i + i0) ** (-gam)
        return w.sum() * (wmax / (i0 ** (-gam)))

    # total(i0) increases with i0: bisection on log i0
    lo, hi = 1e-6, 1e9
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if total(mid) < wsum:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    w = (i + i0) ** (-gam) * (wmax / (i0 ** (-gam)))
    prob = w / w.sum()
    cdf = np.cumsum(prob)
    cdf[-1] = 1.0
    r = rng.random(2 * m_draws)
    ends = np.searchsorted(cdf, r, side="right").astype(np.uint32)
    np.minimum(ends, n - 1, out=ends)
    return n, ends[:m_draws].copy(), ends[m_draws:].copy()


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float,
         seed: int, permute: bool = True):
    """R-MAT (Chakrabarti et al., 2004) with 2**scale vertices and
    edge_factor * 2**scale draws, quadrant probabilities (a, b, c, 1-a-b-c),
    no noise.  Vertex labels are permuted by a seeded random permutation
    (as Graph500 does) so that id locality is not artificially favourable."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor * n
    src = np.zeros(m, np.uint32)
    dst = np.zeros(m, np.uint32)
    ab = a + b
    abc = a + b + c
    for level in range(scale):
        r = rng.random(m, dtype=np.float32)
        bit = np.uint32(1 << (scale - 1 - level))
        # quadrant b: (0,1); c: (1,0); d: (1,1)
        row = r >= ab
        col = ((r >= a) & (r < ab)) | (r >= abc)
        src[row] |= bit
        dst[col] |= bit
    if permute:
        perm = rng.permutation(n).astype(np.uint32)
        src = perm[src]
        dst = perm[dst]
    return n, src, dst


def plant(n: int, src, dst, k: int, p: float, seed: int, exclude=None):
    """Add a G(k, p) block on k distinct random vertices (chosen outside
    ``exclude`` if given).  Returns (n, src, dst, block_vertices)."""
    rng = np.random.default_rng(seed)
    if exclude is None or len(exclude) == 0:
        verts = rng.choice(n, size=k, replace=False).astype(np.uint32)
    else:
        mask = np.ones(n, bool)
        mask[np.asarray(exclude, np.int64)] = False
        pool = np.nonzero(mask)[0]
        verts = rng.choice(pool, size=k, replace=False).astype(np.uint32)
    iu, ju = np.triu_indices(k, 1)
    keep = rng.random(iu.size) < p
    bs = verts[iu[keep]]
    bd = verts[ju[keep]]
    return (n, np.concatenate([np.asarray(src, np.uint32), bs]),
            np.concatenate([np.asarray(dst, np.uint32), bd]), verts)


def concat(*edge_lists):
    s = np.concatenate([np.asarray(e[0], np.uint32) for e in edge_lists])
    d = np.concatenate([np.asarray(e[1], np.uint32) for e in edge_lists])
    return s, d


def random_small(n: int, p: float, seed: int, loops: bool = True,
                 dups: bool = True):
    """Tiny test graphs: G(n, p) plus optional self-loops and repeated /
    reversed pairs, to exercise the builders' clean-up."""
    rng = np.random.default_rng(seed)
    n_, s, d = er(n, p, seed)
    parts_s, parts_d = [s], [d]
    if dups and s.size:
        pick = rng.integers(0, s.size, size=max(1, s.size // 4))
        parts_s += [d[pick], s[pick]]
        parts_d += [s[pick], d[pick]]
    if loops and n > 0:
        lv = rng.integers(0, n, size=max(1, n // 8)).astype(np.uint32)
        parts_s.append(lv)
        parts_d.append(lv)
    s = np.concatenate(parts_s).astype(np.uint32)
    d = np.concatenate(parts_d).astype(np.uint32)
    order = rng.permutation(s.size)
    return n, s[order], d[order]


# ---------------------------------------------------------------------------
# Named workloads.  Recipes (all seeds fixed):
#   er2000     : G(2000, 0.005), seed 0                              (h = 2)
#   cl1m       : Chung-Lu n = 1,000,000, 10,000,000 draws, beta = 2.1,
#                max expected degree 20,000, seed 0; plus one planted
#                G(200, 0.5) block on random vertices, seed 1       (h = 3)
#   rmat22     : R-MAT scale 22, edge factor 16,
#                (a,b,c,d) = (0.57, 0.19, 0.19, 0.05), seed 0        (h = 4, 5)
#   cl4m       : Chung-Lu n = 4,000,000, 64,000,000 draws, beta = 2.2,
#                max expected degree sqrt(sum w), seed 7; plus five planted
#                G(300, 0.4) blocks on disjoint random vertices     (h = 3)
# Scaled-down variants (same recipe, smaller n) serve the parity tests that
# the oracle finishes in seconds (cl50k, rmat14) and kernel profiles whose
# inputs still exceed the 129 MB L2 (rmat21: 2^21 vertices, 2^25 draws).
# ---------------------------------------------------------------------------

def _cl_planted(n, draws, beta, wmax, seed, blocks, wsum=None):
    n, s, d = chung_lu(n, draws, beta, wmax, seed, wsum=wsum)
    used = []
    for j, (k, p) in enumerate(blocks):
        n, s, d, verts = plant(n, s, d, k, p, seed + 1 + j, exclude=used)
        used.extend(verts.tolist())
    return n, s, d


def workload(name: str):
    """Return (n, src, dst, h_list) for a named workload."""
    if name == "er2000":
        n, s, d = er(2000, 0.005, 0)
        return n, s, d, [2]
    if name == "cl1m":
        n, s, d = _cl_planted(1_000_000, 10_000_000, 2.1, 20_000.0, 0,
                              [(200, 0.5)])
        return n, s, d, [3]
    if name == "cl50k":
        n, s, d = _cl_planted(50_000, 500_000, 2.1, 1_000.0, 0, [(60, 0.5)])
        return n, s, d, [3]
    if name == "rmat22":
        n, s, d = rmat(22, 16, 0.57, 0.19, 0.19, 0)
        return n, s, d, [4, 5]
    if name == "rmat14":
        n, s, d = rmat(14, 16, 0.57, 0.19, 0.19, 0)
        return n, s, d, [4, 5]
    if name == "rmat21":
        n, s, d = rmat(21, 16, 0.57, 0.19, 0.19, 0)
        return n, s, d, [4, 5]
    if name == "cl4m":
        draws = 64_000_000
        n, s, d = _cl_planted(4_000_000, draws, 2.2,
                              math.sqrt(2.0 * draws), 7, [(300, 0.4)] * 5)
        return n, s, d, [3]
    raise KeyError(name)


WORKLOADS = ("er2000", "cl1m", "cl50k", "rmat22", "rmat14", "rmat21", "cl4m")


# ---------------------------------------------------------------------------
# Batches of small graphs.  Graph i: seed s_i = splitmix64(1000 + i) (the
# standard 64-bit SplitMix constants), n = clamp(round(exp(N(ln 2000, 1.1^2))),
# 50, 50000); type i mod 3: ER with average degree U[8, 32]; Chung-Lu with
# exponent U[2.0, 2.5] and average degree U[8, 32]; ER background (average
# degree U[8, 32]) plus a planted G(k, 0.6), k uniform in 10..100 (capped at
# n); clique size h uniform in {2, 3, 4}.
# ---------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def batch_graph(i: int, nmax: int = 50000, nmedian: float = 2000.0):
    """Graph i of the mixed batch: (n, src, dst, h)."""
    seed = splitmix64(1000 + i)
    rng = np.random.default_rng(seed)
    n = int(min(max(round(math.exp(rng.normal(math.log(nmedian), 1.1))), 50), nmax))
    avg = float(rng.uniform(8.0, 32.0))
    h = int(rng.integers(2, 5))
    kind = i % 3
    sub = int(rng.integers(0, 2**31))
    if kind == 0:
        _, s, d = er(n, min(1.0, avg / max(n - 1, 1)), sub)
    elif kind == 1:
        beta = float(rng.uniform(2.0, 2.5))
        draws = max(1, int(avg * n / 2))
        wmax = max(2.0, math.sqrt(avg * n))
        _, s, d = chung_lu(n, draws, beta, wmax, sub)
    else:
        _, s, d = er(n, min(1.0, avg / max(n - 1, 1)), sub)
        k = int(min(rng.integers(10, 101), n))
        _, s, d, _ = plant(n, s, d, k, 0.6, sub + 1)
    return n, s, d, h


def batch(count: int = 4096, nmax: int = 50000, nmedian: float = 2000.0):
    return [batch_graph(i, nmax, nmedian) for i in range(count)]


# ---------------------------------------------------------------------------
# Training graphs for the density proposal.  Graph i: seed
# splitmix64(2,000,000 + i) (disjoint from the batch seeds and from the named
# workloads), n = clamp(round(exp(N(ln 3000, 1.2^2))), 50, nmax); type i mod 4:
# ER with average degree U[8, 32]; Chung-Lu with exponent U[2.0, 2.5] and
# average degree U[8, 32]; ER background plus a planted G(k, U[0.4, 0.8]),
# k uniform in 10..150; Chung-Lu background plus 1-5 planted G(k, U[0.3, 0.7])
# blocks on disjoint vertices, k uniform in 20..300 (the shape of the
# cl4m workload).  Clique size h = 3.
# ---------------------------------------------------------------------------

def train_graph(i: int, nmax: int = 200000, nmedian: float = 3000.0):
    """Training graph i: (n, src, dst, h)."""
    seed = splitmix64(2_000_000 + i)
    rng = np.random.default_rng(seed)
    n = int(min(max(round(math.exp(rng.normal(math.log(nmedian), 1.2))), 50), nmax))
    avg = float(rng.uniform(8.0, 32.0))
    kind = i % 4
    sub = int(rng.integers(0, 2**31))
    if kind in (0, 2):
        _, s, d = er(n, min(1.0, avg / max(n - 1, 1)), sub)
    else:
        beta = float(rng.uniform(2.0, 2.5))
        draws = max(1, int(avg * n / 2))
        wmax = max(2.0, math.sqrt(avg * n))
        _, s, d = chung_lu(n, draws, beta, wmax, sub)
    if kind == 2:
        k = int(min(rng.integers(10, 151), n))
        _, s, d, _ = plant(n, s, d, k, float(rng.uniform(0.4, 0.8)), sub + 1)
    elif kind == 3:
        used = []
        for j in range(int(rng.integers(1, 6))):
            k = int(min(rng.integers(20, 301), n - len(used)))
            if k < 3:
                break
            _, s, d, verts = plant(n, s, d, k, float(rng.uniform(0.3, 0.7)), sub + 1 + j,
                                   exclude=used)
            used.extend(verts.tolist())
    return n, s, d, 3


# ---------------------------------------------------------------------------
# Large graphs shaped like the cl4m workload: 16 n Chung-Lu endpoint draws,
# exponent U[2.1, 2.4], maximum expected degree sqrt(32 n), plus 1-5 planted
# G(k, U[0.3, 0.5]) blocks on disjoint vertices, k uniform in 150..300,
# n = round(exp(U[ln nmin, ln nmax])); clique size h = 3.
#   held-out evaluation graph i: seed splitmix64(3,000,000 + i), n in
#     [200,000, 4,000,000], never used in training;
#   large training graph i: seed splitmix64(4,000,000 + i), n in
#     [100,000, 2,000,000].
# Both seed ranges are disjoint from each other, from the small training
# graphs, the batches and the named workloads.
# ---------------------------------------------------------------------------

def _cl_blocks_graph(seed: int, nmin: int, nmax: int):
    rng = np.random.default_rng(seed)
    n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
    beta = float(rng.uniform(2.1, 2.4))
    draws = 16 * n
    sub = int(rng.integers(0, 2**31))
    blocks = [(int(rng.integers(150, 301)), float(rng.uniform(0.3, 0.5)))
              for _ in range(int(rng.integers(1, 6)))]
    n, s, d = _cl_planted(n, draws, beta, math.sqrt(2.0 * draws), sub, blocks)
    return n, s, d, 3


def heldout_graph(i: int, nmin: int = 200_000, nmax: int = 4_000_000):
    """Held-out evaluation graph i: (n, src, dst, h)."""
    return _cl_blocks_graph(splitmix64(3_000_000 + i), nmin, nmax)


def train_large_graph(i: int, nmin: int = 100_000, nmax: int = 2_000_000):
    """Large training graph i: (n, src, dst, h)."""
    return _cl_blocks_graph(splitmix64(4_000_000 + i), nmin, nmax)
