"""Pins of the quality oracle (oracle/quality.py) against closed forms,
brute force and properties the mathematics fixes (no GPU)."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from oracle import checks
from oracle import quality as Q


def _path(n, w=None):
    a = np.arange(n - 1)
    b = a + 1
    return a, b, (np.ones(n - 1) if w is None else np.asarray(w, float))


def _cycle(n):
    a = np.arange(n)
    b = (a + 1) % n
    return np.minimum(a, b), np.maximum(a, b), np.ones(n)


def _random_graph(n, m, rng, connected=True):
    """A random simple graph: a random spanning tree (if connected) plus extra edges."""
    edges = set()
    if connected:
        perm = rng.permutation(n)
        for i in range(1, n):
            x, y = int(perm[i]), int(perm[rng.integers(0, i)])
            edges.add((min(x, y), max(x, y)))
    while len(edges) < m:
        x, y = (int(t) for t in rng.integers(0, n, 2))
        if x != y:
            edges.add((min(x, y), max(x, y)))
    e = np.array(sorted(edges))
    return e[:, 0], e[:, 1], rng.uniform(1.0, 10.0, len(e))


def test_laplacian_rows_sum_to_zero_and_quadratic_form():
    rng = np.random.default_rng(0)
    a, b, w = _random_graph(40, 90, rng)
    L = Q.laplacian_csr(40, a, b, w)
    assert np.abs(L @ np.ones(40)).max() < 1e-12
    x = rng.standard_normal(40)
    assert float(x @ (L @ x)) == pytest.approx(float(np.sum(w * (x[a] - x[b]) ** 2)), rel=1e-12)


def test_laplacian_of_a_path_has_the_cosine_eigenpairs():
    """Unit path P_n: L v_k = (2 - 2 cos(pi k / n)) v_k, v_k(j) = cos(pi k (j + 1/2) / n)."""
    n = 17
    L = Q.laplacian_csr(n, *_path(n))
    j = np.arange(n)
    for k in range(n):
        v = np.cos(np.pi * k * (j + 0.5) / n)
        lam = 2.0 - 2.0 * np.cos(np.pi * k / n)
        assert np.abs(L @ v - lam * v).max() < 1e-12


def test_density_closed_forms():
    assert Q.density(10, 9) == pytest.approx(-0.1)  # a spanning tree: -1/n
    assert Q.density(5, 10) == pytest.approx(1.0)   # K5


def _brute_max_forest(n, a, b, w):
    """Among all edge subsets of size n - c that form a forest, the heaviest."""
    c = checks.n_components(n, list(a), list(b))
    best, best_w = None, -1.0
    for sub in itertools.combinations(range(len(a)), n - c):
        if checks.n_components(n, [a[i] for i in sub], [b[i] for i in sub]) != c:
            continue
        tot = sum(w[i] for i in sub)
        if tot > best_w:
            best, best_w = sub, tot
    return sorted(best)


@pytest.mark.parametrize("seed", range(6))
def test_max_spanning_forest_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 6
    a, b, w = _random_graph(n, 9, rng, connected=seed % 2 == 0)
    w = rng.permutation(len(a)).astype(float) + 1.0  # distinct weights: the forest is unique
    assert list(Q.max_spanning_forest(n, a, b, w)) == _brute_max_forest(n, list(a), list(b), list(w))


def test_laplacian_solver_potential_drop_on_a_path():
    """Unit current from vertex 0 to vertex n-1 through unit resistors drops the
    potential by one per edge."""
    n = 9
    z = Q.LaplacianSolver(n, *_path(n)).solve(np.eye(n)[0] - np.eye(n)[n - 1])
    assert np.abs((z[0] - z) - np.arange(n)).max() < 1e-12


def test_laplacian_solver_two_components():
    rng = np.random.default_rng(3)
    a1, b1, w1 = _random_graph(12, 20, rng)
    a2, b2, w2 = _random_graph(8, 11, rng)
    a = np.concatenate([a1, a2 + 12])
    b = np.concatenate([b1, b2 + 12])
    w = np.concatenate([w1, w2])
    n = 21  # vertex 20 is isolated
    r = rng.standard_normal(n)
    r = Q.project_out_constants(n, a, b, r)
    z = Q.LaplacianSolver(n, a, b, w).solve(r)
    L = Q.laplacian_csr(n, a, b, w)
    assert np.abs(L @ z - r).max() < 1e-10


def test_pcg_exact_preconditioner_takes_one_iteration():
    rng = np.random.default_rng(4)
    n = 60
    g = _random_graph(n, 150, rng)
    bb = Q.project_out_constants(n, g[0], g[1], rng.standard_normal(n))
    x, it, hist = Q.pcg(n, g, bb, h_edges=g, precond="sparsifier")
    assert it == 1 and hist[-1] < 1e-10


def test_cg_on_a_cycle_ends_within_its_distinct_eigenvalues():
    """Unpreconditioned CG on the unit cycle C_n: at most floor(n/2) + 1
    distinct Laplacian eigenvalues, the zero one not excited by b."""
    n = 14
    rng = np.random.default_rng(5)
    g = _cycle(n)
    bb = rng.standard_normal(n)
    bb -= bb.mean()
    _, it, hist = Q.pcg(n, g, bb, precond="none", tol=1e-10)
    assert it <= n // 2 and hist[-1] < 1e-10


def test_jacobi_on_a_regular_graph_equals_plain_cg():
    """On a cycle with unit weights diag(L) = 2 I: the scaled identity changes nothing."""
    n = 30
    rng = np.random.default_rng(6)
    g = _cycle(n)
    bb = rng.standard_normal(n)
    bb -= bb.mean()
    x0, it0, h0 = Q.pcg(n, g, bb, precond="none")
    x1, it1, h1 = Q.pcg(n, g, bb, precond="jacobi")
    assert it0 == it1
    assert np.allclose(h0, h1, rtol=1e-9, atol=0)
    assert np.allclose(x0, x1, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sparsifier_pcg_with_k_missing_edges_takes_at_most_k_plus_one(k):
    """L_G = L_H + (k rank-one terms): the preconditioned operator has at most
    k + 1 distinct eigenvalues, so PCG ends in at most k + 1 iterations."""
    rng = np.random.default_rng(10 + k)
    n = 50
    a, b, w = _random_graph(n, n - 1 + k, rng)
    tree = Q.max_spanning_forest(n, a, b, w)
    h = (a[tree], b[tree], w[tree])
    bb = Q.project_out_constants(n, a, b, rng.standard_normal(n))
    _, it, hist = Q.pcg(n, (a, b, w), bb, h_edges=h, precond="sparsifier", tol=1e-10)
    assert it <= k + 1 and hist[-1] < 1e-10


def test_pcg_solves_and_respects_the_kappa_bound():
    """The result solves L_G x = b, and the iteration count stays within the
    classical bound ceil(sqrt(kappa) / 2 * ln(2 / tol)) + 1 (kappa dense)."""
    rng = np.random.default_rng(7)
    n = 80
    a, b, w = _random_graph(n, 240, rng)
    tree = Q.max_spanning_forest(n, a, b, w)
    rest = np.setdiff1d(np.arange(len(a)), tree)
    keep = np.concatenate([tree, rng.choice(rest, 20, replace=False)])
    h = (a[keep], b[keep], w[keep])
    bb = Q.project_out_constants(n, a, b, rng.standard_normal(n))
    x, it, hist = Q.pcg(n, (a, b, w), bb, h_edges=h, precond="sparsifier")
    xs = np.linalg.pinv(checks.laplacian(n, a, b, w), hermitian=True) @ bb
    assert np.abs(Q.project_out_constants(n, a, b, x) - xs).max() < 1e-6 * np.abs(xs).max()
    kap = checks.kappa(n, (a, b, w), h)
    assert it <= int(np.ceil(np.sqrt(kap) / 2 * np.log(2 / 1e-8))) + 1
    assert hist[-1] < 1e-8


def test_smallest_pencil_eigenvalue_is_one_for_a_subgraph():
    """With H a subgraph of G (same weights) and a vertex untouched by G \\ H,
    the smallest generalized eigenvalue is 1, so kappa = lambda_max."""
    rng = np.random.default_rng(8)
    n = 40
    a, b, w = _random_graph(n, 100, rng)
    tree = Q.max_spanning_forest(n, a, b, w)
    rest = np.setdiff1d(np.arange(len(a)), tree)
    keep = np.concatenate([tree, rest[:10]])
    gone = rest[10:]
    assert len(set(a[gone]) | set(b[gone])) < n  # some vertex keeps all its G edges in H
    ev = checks.pencil_eigs(n, (a, b, w), (a[keep], b[keep], w[keep]))
    assert ev[0] == pytest.approx(1.0, abs=1e-9)
    assert checks.kappa(n, (a, b, w), (a[keep], b[keep], w[keep])) == pytest.approx(ev[-1], rel=1e-9)


def test_forest_potentials_on_a_path_and_against_the_grounded_solve():
    """Unit path: unit current from 0 to n-1 drops the potential by one per
    edge; on random weighted forests the exact potentials solve L_F z = r and
    agree with the grounded sparse solve."""
    n = 9
    z = Q.forest_potentials(n, *_path(n), np.eye(n)[0] - np.eye(n)[n - 1])
    assert np.array_equal(z, -np.arange(n, dtype=float))
    rng = np.random.default_rng(12)
    for trial in range(3):
        n = 60
        a, b, w = _random_graph(n, 90, rng, connected=trial != 1)
        f = Q.max_spanning_forest(n, a, b, w)
        fa, fb, fw = a[f], b[f], w[f]
        r = Q.project_out_constants(n, fa, fb, rng.standard_normal(n))
        z = Q.forest_potentials(n, fa, fb, fw, r)
        L = Q.laplacian_csr(n, fa, fb, fw)
        assert np.abs(L @ z - r).max() < 1e-12
        zr = Q.LaplacianSolver(n, fa, fb, fw).solve(r)
        assert np.abs(z - zr).max() < 1e-10 * np.abs(zr).max()
        lab = checks.components(n, list(fa), list(fb))
        for c in np.unique(lab):
            assert z[np.flatnonzero(lab == c)[0]] == 0.0


def test_pseudo_inverse_apply_matches_pinv():
    """P S P (grounded solves between mean projections) is the Moore-Penrose
    pseudo-inverse, also for right-hand sides with a constant part."""
    rng = np.random.default_rng(13)
    a1, b1, w1 = _random_graph(15, 30, rng)
    a2, b2, w2 = _random_graph(9, 14, rng)
    a = np.concatenate([a1, a2 + 15])
    b = np.concatenate([b1, b2 + 15])
    w = np.concatenate([w1, w2])
    n = 26  # one isolated vertex
    r = rng.standard_normal(n)
    z = Q.LaplacianSolver(n, a, b, w).pinv_apply(r)
    zp = np.linalg.pinv(checks.laplacian(n, a, b, w), hermitian=True) @ r
    assert np.abs(z - zp).max() < 1e-10 * np.abs(zp).max()
