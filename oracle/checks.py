"""Dense FP64 spectral checks and brute-force enumerations for tiny graphs.

TEST INFRASTRUCTURE ONLY (imported by the test suite).  Everything here is a
plain textbook definition that the tests use to pin the oracle:

* Laplacian L = D - A (Section II-A).
* Effective resistance R_eff(p, q) = b_pq^T L^+ b_pq (Definition 1, Eq. 2),
  through the Moore-Penrose pseudo-inverse.
* Relative condition number kappa(L_G, L_H) = lambda_max / lambda_min of the
  pencil (L_G, L_H) restricted to the complement of the all-ones vector
  (Eqs. 6-10), computed by a dense generalized symmetric eigen-solve on the
  Laplacians grounded at one vertex.
* Non-backtracking walk enumeration: every walk of the Section III-B sampler
  with its exact probability, the product of 1 / n_eff over its steps.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def laplacian(n, a, b, w) -> np.ndarray:
    L = np.zeros((n, n))
    for x, y, ww in zip(a, b, w):
        L[x, y] -= ww
        L[y, x] -= ww
        L[x, x] += ww
        L[y, y] += ww
    return L


def effective_resistance(n, a, b, w, p, q) -> float:
    """b_pq^T L^+ b_pq (Definition 1)."""
    Lp = np.linalg.pinv(laplacian(n, a, b, w), hermitian=True)
    bpq = np.zeros(n)
    bpq[p], bpq[q] = 1.0, -1.0
    return float(bpq @ Lp @ bpq)


def effective_resistances(n, a, b, w, pairs) -> np.ndarray:
    Lp = np.linalg.pinv(laplacian(n, a, b, w), hermitian=True)
    out = []
    for p, q in pairs:
        out.append(Lp[p, p] + Lp[q, q] - 2.0 * Lp[p, q])
    return np.asarray(out)


def pencil_eigs(n, g_edges, h_edges) -> np.ndarray:
    """Finite generalized eigenvalues of (L_G, L_H) for connected G, H on the same
    vertex set: grounding one vertex removes the shared all-ones null space."""
    LG = laplacian(n, *g_edges)[1:, 1:]
    LH = laplacian(n, *h_edges)[1:, 1:]
    return sla.eigh(LG, LH, eigvals_only=True)


def kappa(n, g_edges, h_edges) -> float:
    ev = pencil_eigs(n, g_edges, h_edges)
    return float(ev[-1] / ev[0])


def components(n, a, b) -> np.ndarray:
    """Component label per vertex (plain union-find)."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for x, y in zip(a, b):
        rx, ry = find(int(x)), find(int(y))
        if rx != ry:
            parent[rx] = ry
    return np.array([find(x) for x in range(n)])


def n_components(n, a, b) -> int:
    return int(np.unique(components(n, a, b)).size)


def kruskal_max_forest(n, a, b, w):
    """Edge ids of the max-weight spanning forest: scan by (w desc, id asc)."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    order = sorted(range(len(a)), key=lambda i: (-w[i], i))
    out = []
    for i in order:
        rx, ry = find(int(a[i])), find(int(b[i]))
        if rx != ry:
            parent[rx] = ry
            out.append(i)
    return sorted(out)


def adjacency_lists(n, a, b, w):
    """Neighbour lists sorted by id: list of [(nbr, w)]."""
    adj = [[] for _ in range(n)]
    for x, y, ww in zip(a, b, w):
        adj[int(x)].append((int(y), float(ww)))
        adj[int(y)].append((int(x), float(ww)))
    for L in adj:
        L.sort()
    return adj


def enumerate_nb_walks(adj, p, q, T):
    """All walks of the non-backtracking sampler from p (target q, no K).

    A walk stops on reaching q, after T steps, or at a vertex whose only
    neighbour is the one it came from (a leaf).  Returns {path tuple: prob},
    prob = product over steps of 1 / (number of allowed neighbours)."""
    out = {}

    def rec(path, prev, prob):
        c = path[-1]
        steps = len(path) - 1
        if steps > 0 and (c == q or steps == T):
            out[tuple(path)] = out.get(tuple(path), 0.0) + prob
            return
        cand = [y for (y, _) in adj[c] if y != prev]
        if not cand:
            out[tuple(path)] = out.get(tuple(path), 0.0) + prob
            return
        for y in cand:
            rec(path + [y], c, prob / len(cand))

    rec([p], -1, 1.0)
    return out


def tree_path(adj, p, q):
    """The unique p -> q path in a tree (BFS parents)."""
    par = {p: None}
    frontier = [p]
    while frontier:
        nxt = []
        for x in frontier:
            for y, _ in adj[x]:
                if y not in par:
                    par[y] = x
                    nxt.append(y)
        frontier = nxt
    path = [q]
    while path[-1] != p:
        path.append(par[path[-1]])
    return path[::-1]
