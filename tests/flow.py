"""Exact optimal density rho_opt by minimum st-cuts (test helper, small graphs).

Networks (Sec. 3.1):
* h >= 3: Algorithm 1's network -- s->v with capacity deg(v, Psi), v->t with
  capacity alpha*h, psi->v with infinite capacity for v in an (h-1)-clique
  psi, and v->psi with capacity 1 when psi + v is an h-clique.  For a source
  side holding the vertex set A the best cut is
  h*mu(G) - h*mu(A) + alpha*h*|A|, so a cut below h*mu(G) exists exactly
  when some A has mu(A) > alpha*|A|.
* h = 2: Goldberg's network -- s->v capacity m, v->t capacity
  m + 2*alpha - deg(v), and capacity 1 both ways along every edge; its cut
  for A is m*n + 2*(alpha*|A| - e(A)).

alpha = p/q is kept exact by scaling every capacity by q.  Instead of the
paper's binary search with the 1/(n(n-1)) stopping gap (Algorithm 1), the
search is Dinkelbach's iteration alpha <- mu(A)/|A| on the minimising source
side A until no set beats alpha; it visits finitely many densities and ends
at rho_opt exactly.

Dinic's algorithm with Python integers; meant for graphs of at most a few
dozen vertices.
"""
from __future__ import annotations

import itertools
from collections import deque
from fractions import Fraction

import numpy as np


class Dinic:
    def __init__(self, n):
        self.n = n
        self.g = [[] for _ in range(n)]   # edges: [to, cap, rev_index]

    def add(self, u, v, c):
        self.g[u].append([v, c, len(self.g[v])])
        self.g[v].append([u, 0, len(self.g[u]) - 1])

    def _bfs(self, s, t):
        self.level = [-1] * self.n
        self.level[s] = 0
        dq = deque([s])
        while dq:
            u = dq.popleft()
            for v, c, _ in self.g[u]:
                if c > 0 and self.level[v] < 0:
                    self.level[v] = self.level[u] + 1
                    dq.append(v)
        return self.level[t] >= 0

    def _dfs(self, u, t, f):
        if u == t:
            return f
        while self.it[u] < len(self.g[u]):
            e = self.g[u][self.it[u]]
            v, c, r = e
            if c > 0 and self.level[v] == self.level[u] + 1:
                d = self._dfs(v, t, min(f, c))
                if d > 0:
                    e[1] -= d
                    self.g[v][r][1] += d
                    return d
            self.it[u] += 1
        return 0

    def maxflow(self, s, t):
        flow = 0
        inf = float("inf")
        while self._bfs(s, t):
            self.it = [0] * self.n
            while True:
                f = self._dfs(s, t, inf)
                if not f:
                    break
                flow += f
        return flow

    def source_side(self, s):
        seen = [False] * self.n
        seen[s] = True
        dq = deque([s])
        while dq:
            u = dq.popleft()
            for v, c, _ in self.g[u]:
                if c > 0 and not seen[v]:
                    seen[v] = True
                    dq.append(v)
        return seen


def _cliques_in(A, verts, k):
    verts = sorted(verts)
    out = []
    for S in itertools.combinations(verts, k):
        if all(A[a, b] for a, b in itertools.combinations(S, 2)):
            out.append(S)
    return out


def _best_set(A, h, p, q):
    """Vertex set maximising q*mu(S) - p*|S| via one min cut."""
    n = A.shape[0]
    if h == 2:
        m = int(A.sum()) // 2
        deg = A.sum(1)
        s, t = n, n + 1
        D = Dinic(n + 2)
        for v in range(n):
            D.add(s, v, q * m)
            D.add(v, t, q * m + 2 * p - q * int(deg[v]))
            for u in range(n):
                if A[v, u]:
                    D.add(v, u, q)
        D.maxflow(s, t)
        side = D.source_side(s)
        return [v for v in range(n) if side[v]]
    lam = _cliques_in(A, range(n), h - 1)
    hcl = _cliques_in(A, range(n), h)
    deg = [0] * n
    for S in hcl:
        for v in S:
            deg[v] += 1
    s, t = n + len(lam), n + len(lam) + 1
    D = Dinic(n + len(lam) + 2)
    INF = 1 << 62
    for v in range(n):
        D.add(s, v, q * deg[v])
        D.add(v, t, p * h)
    for i, psi in enumerate(lam):
        node = n + i
        for v in psi:
            D.add(node, v, INF)
        pset = set(psi)
        for v in range(n):
            if v not in pset and all(A[v, u] for u in psi):
                D.add(v, node, q)
    D.maxflow(s, t)
    side = D.source_side(s)
    return [v for v in range(n) if side[v]]


def rho_opt(A, h):
    """Exact maximum h-clique density of any vertex subset (Problem 1)."""
    A = np.asarray(A, bool)
    n = A.shape[0]
    if n == 0:
        return Fraction(0), []
    mu_all = len(_cliques_in(A, range(n), h))
    alpha = Fraction(mu_all, n)
    best_set = list(range(n))
    for _ in range(10 * n + 10):
        S = _best_set(A, h, alpha.numerator, alpha.denominator)
        if not S:
            return alpha, best_set
        muS = len(_cliques_in(A, S, h))
        val = Fraction(muS, len(S))
        if val <= alpha:
            return alpha, best_set
        alpha, best_set = val, S
    raise RuntimeError("Dinkelbach iteration did not settle")
