"""Quality of the sparsifier on the device (Section IV): d_H, Laplacian
products, H's maximum spanning forest and its exact solve, PCG with L_H as the
preconditioner and kappa(L_G, L_H), each against the quality oracle.

Tolerances (floating point; the integer results -- forests, counts -- are
compared exactly):
* Laplacian products: a row sums deg + 1 products in another order than
  scipy, so |y - y_ref| <= 4 (deg + 1) eps * (d |x_i| + sum_j w_ij |x_j|).
* Forest solve: z = L_F^+ r through two exact 128-bit fixed-point prefix
  sums (each current and potential rounded once; entries 2^100 below the
  largest are rounded when scaled), against the correctly rounded potentials
  of the correctly rounded currents: within 2 ulp, plus 1e-15 of the largest
  potential where a sum cancels to far below its terms.
* PCG: the iteration count of conjugate gradients in floating point depends
  on rounding well beyond the stopping test: the oracle's PCG, run with
  three preconditioners that equal L_H^+ up to rounding and constants (the
  grounded LU solve; the same followed by removing each component's mean; a
  dense pseudo-inverse), took 71, 74 and 71 iterations on the 32 x 32 grid
  with its initial sparsifier (kappa 175).  So the counts agree within
  max(2, 5 %), the first six relative residuals within 1e-6 (before
  rounding has grown), the true final residual below the tolerance, and the
  solutions within 1e-6.
* kappa: Lanczos on the pencil, run until the largest Ritz value moves by
  less than 1e-12 relative, against a dense generalized eigen-solve: 1e-7.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import checks
from oracle import quality as Q
from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def _assert_potentials(z, zr):
    """Against the correctly rounded potentials: within 2 ulp, plus 1e-15 of
    the largest potential for sums that cancel to far below it."""
    err = np.abs(z - zr)
    bound = 4 * EPS * np.abs(zr) + 1e-15 * np.abs(zr).max()
    assert np.all(err <= bound), (err.max(), np.argmax(err - bound))


def _graph(name):
    if name == "grid":
        wl, st = W.make_grid(32, 32, seed=1)
    elif name == "mesh":
        wl, st = W.make_mesh3d(10, 10, 10, seed=2)
    elif name == "rmat":
        wl, st = W.make_rmat(11, 12_000, seed=3)  # unit weights: every comparison of weights ties
    else:
        raise ValueError(name)
    return wl, st


def _loaded(name, batches=1, size=(300, 200)):
    wl, st = _graph(name)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for _ in range(batches):
        bt = st.next_batch(*size)
        g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    return wl, ctx, g


@pytest.mark.parametrize("name", ["grid", "mesh", "rmat"])
def test_density_and_laplacian_products(name):
    wl, ctx, g = _loaded(name)
    ga, gb, gw = g.edges()
    ha, hb, hw = g.sparsifier()
    d, mg, mh = g.density()
    assert (mg, mh) == (ga.size, ha.size)
    assert d == Q.density(wl.n, ha.size)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(wl.n)
    dx = _dev(x)
    dy = torch.empty_like(dx)
    for which, (a, b, w) in ((D.LAP_G, (ga, gb, gw)), (D.LAP_H, (ha, hb, hw))):
        g.laplacian_apply(which, dx.data_ptr(), dy.data_ptr())
        torch.cuda.synchronize()
        L = Q.laplacian_csr(wl.n, a, b, w)
        ref = L @ x
        absL = abs(L)
        bound = 4 * (np.diff(L.indptr) + 1) * EPS * (absL @ np.abs(x))
        assert np.all(np.abs(dy.cpu().numpy() - ref) <= bound + 1e-300), which
    ctx.close()


@pytest.mark.parametrize("name", ["grid", "mesh", "rmat"])
def test_forest_is_the_maximum_spanning_forest_of_h(name):
    wl, ctx, g = _loaded(name)
    ha, hb, hw = g.sparsifier()
    ids = Q.max_spanning_forest(wl.n, ha, hb, hw)
    fu, fv = g.debug_sparsifier_forest()
    assert np.array_equal(fu, ha[ids]) and np.array_equal(fv, hb[ids])
    ctx.close()


def test_forest_with_several_trees_and_isolated_vertices():
    """H made of two separate pieces and untouched vertices: one tree each."""
    wl, _ = W.make_grid(20, 20, seed=4)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    keep = (wl.a < 150) | (wl.a >= 250)
    keep &= (wl.b < 150) | (wl.b >= 250)
    keep &= ~((wl.a < 200) & (wl.b >= 200))
    sel = np.flatnonzero(keep)[::2]
    g.init_sparsifier(wl.a[sel], wl.b[sel])
    ha, hb, hw = g.sparsifier()
    ids = Q.max_spanning_forest(wl.n, ha, hb, hw)
    fu, fv = g.debug_sparsifier_forest()
    assert np.array_equal(fu, ha[ids]) and np.array_equal(fv, hb[ids])
    # the forest solve on that forest
    rng = np.random.default_rng(1)
    r = Q.project_out_constants(wl.n, ha[ids], hb[ids], rng.standard_normal(wl.n))
    dr = _dev(r)
    dz = torch.empty_like(dr)
    g.debug_forest_solve(dr.data_ptr(), dz.data_ptr())
    z = dz.cpu().numpy()
    zr = Q.forest_potentials(wl.n, ha[ids], hb[ids], hw[ids], r)
    _assert_potentials(z, zr)
    ctx.close()


@pytest.mark.parametrize("name", ["grid", "mesh", "rmat"])
def test_forest_solve_is_exact(name):
    wl, ctx, g = _loaded(name)
    ha, hb, hw = g.sparsifier()
    ids = Q.max_spanning_forest(wl.n, ha, hb, hw)
    fa, fb, fw = ha[ids], hb[ids], hw[ids]
    rng = np.random.default_rng(2)
    r = Q.project_out_constants(wl.n, fa, fb, rng.standard_normal(wl.n))
    dr = _dev(r)
    dz = torch.empty_like(dr)
    g.debug_forest_solve(dr.data_ptr(), dz.data_ptr())
    z = dz.cpu().numpy()
    # z = 0 at the smallest vertex of every tree
    lab = checks.components(wl.n, list(fa), list(fb))
    for c in np.unique(lab):
        assert z[np.flatnonzero(lab == c)[0]] == 0.0
    _assert_potentials(z, Q.forest_potentials(wl.n, fa, fb, fw, r))
    ctx.close()


@pytest.mark.parametrize("name", ["grid", "mesh", "rmat"])
@pytest.mark.parametrize("precond", ["none", "jacobi", "sparsifier"])
def test_pcg_matches_oracle(name, precond):
    wl, ctx, g = _loaded(name)
    ga, gb, gw = g.edges()
    ha, hb, hw = g.sparsifier()
    rng = np.random.default_rng(3)
    b = Q.project_out_constants(wl.n, ga, gb, rng.standard_normal(wl.n))
    db = _dev(b)
    dx = torch.empty_like(db)
    info, hist = g.pcg_solve(db.data_ptr(), dx.data_ptr(), tol=1e-8, max_iter=5000, precond=precond,
                             inner_tol=1e-13, inner_max_iter=20000)
    xr, itr, hr = Q.pcg(wl.n, (ga, gb, gw), b, h_edges=(ha, hb, hw), precond=precond, tol=1e-8, max_iter=5000)
    assert info["converged"] == 1
    assert abs(info["iters"] - itr) <= max(2, int(np.ceil(0.05 * itr))), (info["iters"], itr)
    assert info["rel_residual"] < 1.5e-8
    k = min(6, itr, info["iters"])
    assert np.allclose(hist[:k + 1], hr[:k + 1], rtol=1e-6, atol=0)
    x = Q.project_out_constants(wl.n, ga, gb, dx.cpu().numpy())
    xr = Q.project_out_constants(wl.n, ga, gb, xr)
    assert np.abs(x - xr).max() <= 1e-6 * np.abs(xr).max()
    if precond == "sparsifier":
        assert info["inner_unconverged"] == 0 and info["inner_iters"] > 0
    ctx.close()


def test_pcg_with_h_equal_g_takes_one_iteration():
    wl, _ = W.make_grid(24, 24, seed=5)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a, wl.b)
    rng = np.random.default_rng(4)
    b = Q.project_out_constants(wl.n, wl.a, wl.b, rng.standard_normal(wl.n))
    db = _dev(b)
    dx = torch.empty_like(db)
    info, _ = g.pcg_solve(db.data_ptr(), dx.data_ptr(), precond="sparsifier", inner_tol=1e-13)
    assert info["iters"] == 1 and info["rel_residual"] < 1e-8
    ctx.close()


@pytest.mark.parametrize("name", ["grid", "mesh"])
def test_kappa_matches_dense_pencil(name):
    """Connected graphs (the R-MAT graph has isolated vertices and many
    components: the next test covers it)."""
    wl, ctx, g = _loaded(name)
    ga, gb, gw = g.edges()
    ha, hb, hw = g.sparsifier()
    lab = checks.components(wl.n, list(ga), list(gb))
    # the dense check grounds one vertex: run it on G's largest component
    big = np.bincount(lab).argmax()
    verts = np.flatnonzero(lab == big)
    assert verts.size == wl.n, "the dense check needs a connected G"
    ref = checks.kappa(wl.n, (ga, gb, gw), (ha, hb, hw))
    v0 = np.random.default_rng(5).standard_normal(wl.n)
    dv = _dev(v0)
    info = g.condition_number(max_iter=min(wl.n, 600), check_every=5, tol=1e-12, inner_tol=1e-13, d_v0=dv.data_ptr())
    assert info["converged"] == 1
    assert info["kappa"] == pytest.approx(ref, rel=1e-7)
    assert info["lambda_min"] >= 1.0 - 1e-8
    ctx.close()


def test_kappa_on_several_components():
    """R-MAT leaves isolated vertices and small components: kappa is taken
    over all of them (the dense check works block by block)."""
    wl, ctx, g = _loaded("rmat")
    ga, gb, gw = g.edges()
    ha, hb, hw = g.sparsifier()
    lab = checks.components(wl.n, list(ga), list(gb))
    ref = 1.0
    for c in np.unique(lab):
        verts = np.flatnonzero(lab == c)
        if verts.size < 2:
            continue
        remap = -np.ones(wl.n, np.int64)
        remap[verts] = np.arange(verts.size)
        ge = np.isin(ga, verts)
        he = np.isin(ha, verts)
        ref = max(ref, checks.kappa(verts.size, (remap[ga[ge]], remap[gb[ge]], gw[ge]),
                                    (remap[ha[he]], remap[hb[he]], hw[he])))
    info = g.condition_number(max_iter=600, check_every=5, tol=1e-12, inner_tol=1e-13, seed=7)
    assert info["kappa"] == pytest.approx(ref, rel=1e-7)
    ctx.close()


def test_h_that_does_not_span_g():
    wl, _ = W.make_grid(16, 16, seed=6)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[:100], wl.b[:100])
    assert g.condition_number(max_iter=10)["kappa"] == np.inf
    db = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DgError) as e:
        g.pcg_solve(db.data_ptr(), db.data_ptr(), precond="sparsifier")
    assert e.value.code == -5
    ctx.close()


def test_quality_follows_the_oracle_stream():
    """d_H after each batch equals the oracle's, batch by batch."""
    wl, st = W.make_mesh3d(10, 10, 10, seed=7)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for _ in range(3):
        bt = st.next_batch(200, 100)
        g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        o.apply(bt.u, bt.v, bt.w, bt.op)
        assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
        assert g.density()[0] == Q.density(wl.n, o.edges("H")[0].size)
    o.close()
    ctx.close()


def test_quality_degenerate_inputs():
    """A zero right-hand side takes no iteration; a graph with no edges has
    kappa 1 and density -1; a single-edge graph with H = G has kappa 1."""
    ctx = D.Context()
    g = ctx.load_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    g.init_sparsifier(np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.density()[0] == -1.0
    k = g.condition_number(max_iter=5)
    assert k["kappa"] == 1.0
    db = torch.zeros(5, dtype=torch.float64, device="cuda")
    dx = torch.empty_like(db)
    info, hist = g.pcg_solve(db.data_ptr(), dx.data_ptr(), precond="none")
    assert info["iters"] == 0 and info["converged"] == 1
    g2 = ctx.load_graph(2, np.array([0], np.int32), np.array([1], np.int32), np.array([2.0]))
    g2.init_sparsifier(np.array([0], np.int32), np.array([1], np.int32))
    assert g2.condition_number(max_iter=5)["kappa"] == pytest.approx(1.0)
    b = _dev(np.array([1.0, -1.0]))
    x = torch.empty_like(b)
    info, _ = g2.pcg_solve(b.data_ptr(), x.data_ptr(), precond="sparsifier")
    assert info["iters"] == 1
    xs = x.cpu().numpy()
    assert (xs[0] - xs[1]) == pytest.approx(0.5)  # unit current through resistance 1/2
    ctx.close()
