"""Brute force over all vertex subsets (n <= 16), written straight from the
definitions, for pinning the oracle.

* clique instances: every h-subset whose pairs are all edges (Def. 2);
* clique-degree and mu (Defs. 3, 4);
* core(v) = max over subsets S containing v of min_{u in S} deg_{G[S]}(u):
  R_k is the largest S whose every vertex has >= k instances inside G[S]
  (Def. 6), and the union of two such sets is again one, so v is in R_k
  exactly when some S containing v has that property;
* rho_opt = max over non-empty S of mu(G[S]) / |S| (Problem 1).
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def adjacency(n, off, adj):
    A = np.zeros((n, n), bool)
    for v in range(n):
        for j in range(int(off[v]), int(off[v + 1])):
            A[v, int(adj[j])] = True
    return A


def cliques(A, h):
    n = A.shape[0]
    out = []
    for S in itertools.combinations(range(n), h):
        if all(A[a, b] for a, b in itertools.combinations(S, 2)):
            out.append(S)
    return out


def clique_degrees(A, h):
    n = A.shape[0]
    deg = np.zeros(n, np.int64)
    cl = cliques(A, h)
    for S in cl:
        for v in S:
            deg[v] += 1
    return deg, len(cl)


def _subset_tables(A, h):
    n = A.shape[0]
    cl = cliques(A, h)
    subsets = np.arange(1 << n, dtype=np.int64)
    if cl:
        cm = np.array([sum(1 << v for v in S) for S in cl], np.int64)
        inside = (subsets[:, None] & cm[None, :]) == cm[None, :]
        member = np.zeros((len(cl), n), np.int64)
        for i, S in enumerate(cl):
            member[i, list(S)] = 1
        degS = inside.astype(np.int64) @ member          # [subsets, n]
        muS = inside.sum(1)
    else:
        degS = np.zeros((subsets.size, n), np.int64)
        muS = np.zeros(subsets.size, np.int64)
    inS = ((subsets[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)
    return subsets, inS, degS, muS


def core_numbers(A, h):
    n = A.shape[0]
    if n == 0:
        return np.zeros(0, np.int64)
    subsets, inS, degS, muS = _subset_tables(A, h)
    big = np.iinfo(np.int64).max
    mins = np.where(inS, degS, big).min(1)
    core = np.zeros(n, np.int64)
    for v in range(n):
        sel = inS[:, v]
        core[v] = mins[sel].max()
    return core


def rho_opt(A, h):
    n = A.shape[0]
    if n == 0:
        return Fraction(0)
    subsets, inS, degS, muS = _subset_tables(A, h)
    size = inS.sum(1)
    best = Fraction(0)
    for s in range(1, n + 1):
        sel = size == s
        best = max(best, Fraction(int(muS[sel].max()), s))
    return best
