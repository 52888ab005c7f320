"""Sequential semantics (Algorithm 1 one update at a time) on the device:
the stream cut into prefixes whose batched execution provably equals the
one-at-a-time execution.  Every result (all bytes the oracle defines), G and H
must equal the oracle's one-update-per-batch run, and the prefixes must be
real batches (fewer batches than updates)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal, assert_results_equal

pytestmark = pytest.mark.gpu


def _pair(wl, **kw):
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s, **kw)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    return ctx, g, o


@pytest.mark.parametrize("name,sizes", [("grid", (300, 200)), ("mesh", (600, 400)), ("rmat", (300, 200))])
def test_sequential_equals_one_update_at_a_time(name, sizes):
    if name == "grid":
        wl, st = W.make_grid(40, 40, seed=21)
    elif name == "mesh":
        wl, st = W.make_mesh3d(16, 16, 16, seed=22)
    else:
        wl, st = W.make_rmat(12, 30_000, seed=23)
    ctx, g, o = _pair(wl)
    total_pre = 0
    for b in range(2):
        bt = st.next_batch(*sizes)
        res, pre = g.apply_sequential(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        ref = o.apply_sequential(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
        assert_results_equal(res, ref, f"{name} batch {b}")
        assert_edges_equal(g.sparsifier(), o.edges("H"), f"{name} H after batch {b}")
        assert_edges_equal(g.edges(), o.edges("G"), f"{name} G after batch {b}")
        assert 1 <= pre < len(bt.u)
        total_pre += pre
    o.close()
    ctx.close()


def test_sequential_with_repeated_edges_and_invalid_updates():
    """Insert-then-delete of one edge, deletions of H edges right after their
    insertion, invalid records: each sees the state its predecessors left."""
    wl, st = W.make_grid(24, 24, seed=24)
    ctx, g, o = _pair(wl)
    bt = st.next_batch(60, 40)
    u, v, w, op = (list(x) for x in (bt.u, bt.v, bt.w, bt.op))
    # the first insertion deleted again, and inserted a third time
    u += [bt.u[0], bt.u[0], 5, 7, -1]
    v += [bt.v[0], bt.v[0], 5, 3, 2]
    w += [1.0, 2.5, 1.0, -1.0, 1.0]
    op += [D.OP_DELETE, D.OP_INSERT, D.OP_INSERT, D.OP_INSERT, D.OP_INSERT]
    u, v, w, op = (np.asarray(x) for x in (u, v, w, op))
    res, pre = g.apply_sequential(D.make_updates(u, v, w, op))
    ref = o.apply_sequential(u.astype(np.int32), v.astype(np.int32), w.astype(np.float64), op.astype(np.int32),
                             prune_bounds=True)
    assert_results_equal(res, ref, "repeats")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert_edges_equal(g.edges(), o.edges("G"), "G")
    o.close()
    ctx.close()


def test_sequential_then_batched_share_the_id_counter():
    """Update ids continue across the two forms: a batch after a sequential run
    gets the same results as on a graph that ran everything one at a time."""
    wl, st = W.make_grid(32, 32, seed=25)
    ctx, g, o = _pair(wl)
    b1 = st.next_batch(200, 100)
    g.apply_sequential(D.make_updates(b1.u, b1.v, b1.w, b1.op))
    o.apply_sequential(b1.u, b1.v, b1.w, b1.op, prune_bounds=True)
    b2 = st.next_batch(200, 100)
    res = g.apply(D.make_updates(b2.u, b2.v, b2.w, b2.op))
    ref = o.apply(b2.u, b2.v, b2.w, b2.op, prune_bounds=True)
    assert_results_equal(res, ref, "batch after sequential")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    o.close()
    ctx.close()


def test_interacting_updates_differ_from_the_snapshot():
    """A small grid where the updates crowd together: the batch snapshot and
    the one-at-a-time order give different results, and the sequential mode
    follows the one-at-a-time order."""
    wl, st = W.make_grid(12, 12, seed=26)
    bt = st.next_batch(80, 60)
    snap = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    snap.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    ref_snap = snap.apply(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
    h_snap = snap.edges("H")
    snap.close()
    ctx, g, o = _pair(wl)
    ref = o.apply_sequential(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
    differs = any(not np.array_equal(np.asarray(ref[f]), np.asarray(ref_snap[f]))
                  for f in ("accepted", "hit", "nrecovered", "steps_lo")) or h_snap[0].size != o.edges("H")[0].size
    assert differs, "the stream does not tell the two orders apart"
    res, pre = g.apply_sequential(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    assert_results_equal(res, ref, "crowded")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert_edges_equal(g.edges(), o.edges("G"), "G")
    assert pre > 1
    o.close()
    ctx.close()


@pytest.mark.parametrize("kw", [dict(early_exit=False), dict(del_prune=False)])
def test_sequential_without_cuts_or_pruning(kw):
    """Without the batch's early exits or pruning every walker runs to its
    end; the prefixes must account for all it reads."""
    wl, st = W.make_grid(20, 20, seed=27)
    ctx, g, o = _pair(wl, **kw)
    if "early_exit" in kw:
        o.close()
        o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s, early_exit=False)
        o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    bt = st.next_batch(120, 80)
    res, pre = g.apply_sequential(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    ref = o.apply_sequential(bt.u, bt.v, bt.w, bt.op, prune_bounds=g.ctx.del_prune)
    assert_results_equal(res, ref, str(kw))
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    o.close()
    ctx.close()


def test_sequential_empty_and_single_update():
    wl, st = W.make_grid(10, 10, seed=28)
    ctx, g, o = _pair(wl)
    res, pre = g.apply_sequential(D.make_updates([], [], [], []))
    assert len(res) == 0 and pre == 0
    bt = st.next_batch(1, 0)
    res, pre = g.apply_sequential(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    ref = o.apply_sequential(bt.u, bt.v, bt.w, bt.op, prune_bounds=True)
    assert pre == 1
    assert_results_equal(res, ref, "single")
    o.close()
    ctx.close()
