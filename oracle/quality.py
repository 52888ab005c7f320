"""Quality measures of a sparsifier, plain and slow (numpy / scipy on the CPU).

TEST INFRASTRUCTURE ONLY: imported by the test suite and the benchmark's
quality line; the product path never loads it.

What the paper measures a sparsifier H of G by (Section IV):

* the off-tree density d_H = |E_H| / |V| - 1 (Section IV, Tables II-IV);
* the relative condition number kappa(L_G, L_H) (Eqs. 6-10; with H a subgraph
  of G it is the largest generalized eigenvalue of the pencil, since the
  smallest is 1) -- ``oracle.checks.kappa`` computes it densely;
* the iterations of the preconditioned conjugate gradient method on
  L_G x = b with L_H as the preconditioner, run until the relative residual
  norm falls below 1e-8 (Section IV, Table IV).

Each function below is the textbook definition:

* ``laplacian_csr``: L = D - A (Section II-A) as a scipy sparse matrix.
* ``max_spanning_forest``: the maximum-weight spanning forest (edges scanned by
  weight descending, then edge id ascending; union-find), the tree a
  preconditioner of L_H is built on.
* ``pcg``: the preconditioned conjugate gradient method in its textbook form
  (Hestenes-Stiefel with a preconditioner, as in Saad, Iterative Methods for
  Sparse Linear Systems, Algorithm 9.1): x0 = 0, r0 = b, z0 = M^-1 r0,
  p0 = z0; alpha = (r, z) / (A p, p); x += alpha p; r -= alpha A p;
  stop when ||r|| / ||b|| < tol; z = M^-1 r; beta = (r_new, z_new) / (r, z);
  p = z + beta p.  M^-1 is exact: for M = L_H it is the pseudo-inverse
  L_H^+ = P S P, with S the solve of every component's Laplacian grounded at
  its smallest vertex (a sparse LU factorization, scipy's SuperLU) and P the
  projection that removes the mean of every component.
* ``forest_potentials``: the exact solve of a forest Laplacian, L_F z = r, in
  its physical reading: with every tree rooted at its smallest vertex
  (z = 0 there), the current through the edge (parent(y), y) is the sum of r
  over y's subtree and z_y is the sum of current / weight over the edges of
  y's root path.  Both sums are taken exactly (rational arithmetic) and
  rounded once, and the division once, so the result is the correctly
  rounded potential of the correctly rounded currents.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.checks import components, kruskal_max_forest


def laplacian_csr(n, a, b, w) -> sp.csr_matrix:
    """L = D - A of the undirected weighted graph with edges (a[i], b[i], w[i])."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    w = np.asarray(w, np.float64)
    A = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([a, b]), np.concatenate([b, a]))), shape=(n, n))
    A = A.tocsr()
    D = sp.diags(np.asarray(A.sum(axis=1)).ravel())
    return (D - A).tocsr()


def density(n: int, m_h: int) -> float:
    """Off-tree density d_H = |E_H| / |V| - 1 (Section IV)."""
    return m_h / n - 1.0


def max_spanning_forest(n, a, b, w) -> np.ndarray:
    """Edge ids (ascending) of the maximum-weight spanning forest, ties by edge id."""
    return np.asarray(kruskal_max_forest(n, list(a), list(b), list(w)), np.int64)


class LaplacianSolver:
    """Exact solve of L z = r for a graph Laplacian: each component grounded at
    its smallest vertex (z = 0 there) and factored once."""

    def __init__(self, n, a, b, w):
        L = laplacian_csr(n, a, b, w).tocsc()
        lab = components(n, list(a), list(b))
        self.n = n
        self.parts = []
        self.comps = []
        for c in np.unique(lab):
            verts = np.flatnonzero(lab == c)  # ascending: verts[0] is the smallest vertex
            self.comps.append(verts)
            rest = verts[1:]
            if rest.size == 0:
                continue
            sub = L[rest][:, rest].tocsc()
            self.parts.append((rest, spla.splu(sub)))

    def solve(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros(self.n)
        for rest, lu in self.parts:
            z[rest] = lu.solve(r[rest])
        return z

    def pinv_apply(self, r: np.ndarray) -> np.ndarray:
        """L^+ r: with P the projection that removes the mean of every
        component and S the grounded solve, L^+ = P S P."""
        return self._center(self.solve(self._center(np.asarray(r, np.float64))))

    def _center(self, v):
        y = v.copy()
        for verts in self.comps:
            y[verts] -= y[verts].mean()
        return y


def pcg(n, g_edges, b, *, h_edges=None, precond="sparsifier", tol=1e-8, max_iter=10_000):
    """Preconditioned CG on L_G x = b (x0 = 0).  precond: "none" (M = I),
    "jacobi" (M = diag(L_G)) or "sparsifier" (M = L_H, exact).  Returns
    (x, iterations, relative residual history [||r_0||/||b||, ...])."""
    A = laplacian_csr(n, *g_edges)
    b = np.asarray(b, np.float64)
    if precond == "none":
        def minv(r):
            return r.copy()
    elif precond == "jacobi":
        d = A.diagonal().copy()
        d[d == 0] = 1.0

        def minv(r):
            return r / d
    elif precond == "sparsifier":
        S = LaplacianSolver(n, *h_edges)

        def minv(r):
            return S.pinv_apply(r)
    else:
        raise ValueError(precond)
    x = np.zeros(n)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(r)) / nb if nb else 0.0]
    if nb == 0.0:
        return x, 0, hist
    z = minv(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < max_iter:
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / nb
        hist.append(rel)
        if rel < tol:
            break
        z = minv(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist


def forest_potentials(n, a, b, w, r) -> np.ndarray:
    """z with L_F z = r on the forest (a, b, w), z = 0 at each tree's smallest vertex."""
    from fractions import Fraction
    adj = [[] for _ in range(n)]
    for x, y, ww in zip(a, b, w):
        adj[int(x)].append((int(y), float(ww)))
        adj[int(y)].append((int(x), float(ww)))
    parent = [-1] * n
    pw = [0.0] * n
    seen = [False] * n
    order = []  # every vertex after its parent
    for s in range(n):  # the first vertex met of each tree is its smallest
        if seen[s]:
            continue
        seen[s] = True
        stack = [s]
        while stack:
            x = stack.pop()
            order.append(x)
            for y, ww in adj[x]:
                if not seen[y]:
                    seen[y] = True
                    parent[y] = x
                    pw[y] = ww
                    stack.append(y)
    sub = [Fraction(float(v)) for v in r]
    for x in reversed(order):
        if parent[x] >= 0:
            sub[parent[x]] += sub[x]
    pot = [Fraction(0)] * n
    z = np.zeros(n)
    for x in order:
        p = parent[x]
        if p >= 0:
            a_x = float(sub[x]) / pw[x]
            pot[x] = pot[p] + Fraction(a_x)
            z[x] = float(pot[x])
    return z


def project_out_constants(n, a, b, x) -> np.ndarray:
    """x minus its mean on every component of the graph (a, b)."""
    lab = components(n, list(a), list(b))
    y = np.asarray(x, np.float64).copy()
    for c in np.unique(lab):
        idx = lab == c
        y[idx] -= y[idx].mean()
    return y
