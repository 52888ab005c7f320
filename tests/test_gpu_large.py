"""Parity on the large synthetic workloads.

* FEA-like triangulated 2048 x 2048 grid (4.2M vertices, 12.6M edges) at its
  full batch of 100k mixed updates, in the benchmark's launch form (the first
  batch autotunes, the second replays the captured step): every update result
  and the final H and G match the oracle.
* R-MAT scale 22 (4.2M vertices, 64M edges, power law with hubs of degree
  > 10^5, 1.8M isolated vertices): two full batches of 50k updates (60 %
  insertions between random vertices, 40 % deletions of current edges), the
  benchmark's workload and launch form; every update result, H and G match
  the oracle, which runs the walks of a batch on every host core (its OpenMP
  build, identical to the single-threaded one).  Scale 18 runs the same way
  in a few seconds.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal, assert_results_equal, pair, step_both

pytestmark = pytest.mark.gpu


def test_fea_full_size_batches():
    wl, st = W.make_fea()
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    for bi in range(2):
        bt = st.next_batch(50_000, 50_000)
        res, _ = step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"fea batch {bi}")
        assert (res["status"] == 0).all()
    assert g.stats()["graph_replayed"] == 1
    ctx.close()


def _rmat_full(scale, n_edges, n_ins, n_del, batches=2):
    wl, st = W.make_rmat(scale, n_edges)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s, threads=0)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for bi in range(batches):
        bt = st.next_batch(n_ins, n_del)
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        ref = o.apply(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
        assert_results_equal(res, ref, f"rmat s{scale} batch {bi}")
        assert (res["status"] == 0).all() and res["walked"].sum() > 0
        assert (res["walked"].astype(bool) & (res["steps"] == 0)).any()  # isolated starts walk 0 steps
        assert res["fallback"].sum() > 0 and res["hit"].sum() > 0
    assert g.stats()["graph_replayed"] == 1
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert_edges_equal(g.edges(), o.edges("G"), "G")
    o.close()
    ctx.close()


def test_rmat_scale18_full_batches():
    _rmat_full(18, 4_000_000, 12_000, 8_000)


def test_rmat_scale22_full_size():
    """The power-law configuration at full size: 64M edges, 50k-update batches."""
    _rmat_full(22, 64_000_000, 30_000, 20_000)


def test_mesh_full_size_sequential_batch():
    """Sequential semantics at the mesh configuration's full batch (10k + 10k
    on the 100^3 mesh): every result, H and G equal the oracle applying the
    updates one per batch."""
    wl, st = W.make_mesh3d(100, 100, 100)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    bt = st.next_batch(10_000, 10_000)
    res, pre = g.apply_sequential(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    ref = o.apply_sequential(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
    assert_results_equal(res, ref, "mesh sequential")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert_edges_equal(g.edges(), o.edges("G"), "G")
    assert 1 < pre < 20_000
    o.close()
    ctx.close()


def test_rmat_scale22_sequential_prefix():
    """Sequential semantics on the power-law configuration at full size (64M
    edges): the first 4000 updates of a batch, one at a time."""
    wl, st = W.make_rmat(22, 64_000_000)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    bt = st.next_batch(30_000, 20_000)
    k = 4000
    u, v, w, op = bt.u[:k], bt.v[:k], bt.w[:k], bt.op[:k]
    res, pre = g.apply_sequential(D.make_updates(u, v, w, op))
    ref = o.apply_sequential(u, v, w, op, prune_bounds=True)
    assert_results_equal(res, ref, "rmat sequential")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert 1 < pre < k
    o.close()
    ctx.close()


def test_quality_properties_at_full_size():
    """The quality calls on the mesh configuration at full size, by the
    properties that hold at any size.  After an insertion batch (the paper's
    quality experiment): PCG's recomputed residual is below its tolerance and
    kappa >= the smallest Ritz value >= 1 (H is a subgraph of G).  After a
    mixed batch: kappa is infinite exactly when H has more connected
    components than G (a deletion whose walkers all missed keeps only the
    fallback edges at its endpoints, which need not reconnect H)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    import torch
    wl, st = W.make_mesh3d(100, 100, 100)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    bt = st.next_batch(25_000, 0)
    g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    rng = np.random.default_rng(0)
    b = rng.standard_normal(wl.n)
    b -= b.mean()
    db = torch.from_numpy(b).cuda()
    dx = torch.empty_like(db)
    info, hist = g.pcg_solve(db.data_ptr(), dx.data_ptr(), tol=1e-8, max_iter=2000, inner_tol=1e-10)
    assert info["converged"] == 1 and info["rel_residual"] < 1.5e-8
    k = g.condition_number(max_iter=300, check_every=10, tol=1e-6, inner_tol=1e-10)
    assert k["converged"] == 1 and k["kappa"] >= k["lambda_min"] >= 1.0 - 1e-6

    def ncomp(edges):
        a_, b_, _ = edges
        m = sp.coo_matrix((np.ones(a_.size), (a_, b_)), shape=(wl.n, wl.n))
        return connected_components(m, directed=False)[0]

    bt = st.next_batch(10_000, 10_000)
    g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    spans = ncomp(g.sparsifier()) == ncomp(g.edges())
    k = g.condition_number(max_iter=300, check_every=10, tol=1e-6, inner_tol=1e-10)
    assert (k["kappa"] == np.inf) == (not spans)
    ctx.close()
