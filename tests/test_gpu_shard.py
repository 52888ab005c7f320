"""Sharded batches over replicas (Section III-F: a batch's walked updates are
independent walk tasks on one snapshot).

Two or three contexts on this GPU stand in for replicas on separate GPUs:
each holds the same G and H, walks its contiguous share of the batch's walked
updates, exports one record per walked update, and commits the gathered
records of every replica.  Every replica's results, H and G must equal,
byte for byte, the unsharded batch and the oracle.  The replicas exchange
records through the host only; no kernel of one waits on another.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal, assert_results_equal, assert_same_outputs

pytestmark = pytest.mark.gpu


def _graphs(wl, k, **kw):
    out = []
    for _ in range(k):
        ctx = D.Context(K=wl.K, T=wl.T, s=wl.s, **kw)
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        out.append((ctx, g))
    return out


def _sharded(replicas, ups, rng):
    world = len(replicas)
    counts = [g.shard_begin(ups, r, world) for r, (_, g) in enumerate(replicas)]
    recs = np.concatenate([g.shard_export() for _, g in replicas])
    assert len(recs) == sum(counts)
    recs = recs[rng.permutation(len(recs))]  # gathered in any order
    return [g.shard_commit(recs) for _, g in replicas], counts


@pytest.mark.parametrize("world,del_prune", [(2, True), (3, True), (2, False)])
def test_sharded_batches_match_unsharded_and_oracle(world, del_prune):
    wl, st = W.make_grid(40, 40)
    rng = np.random.default_rng(world)
    reps = _graphs(wl, world, del_prune=del_prune)
    (ctx1, g1), = _graphs(wl, 1, del_prune=del_prune)
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for bi in range(4):
        bt = st.next_batch(300, 250)
        ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
        outs, counts = _sharded(reps, ups, rng)
        ref = g1.apply(ups)
        assert min(counts) > 0 and sum(counts) == int(ref["walked"].sum())
        for r in outs:
            assert_same_outputs(r, ref)
        assert_results_equal(ref, o.apply(bt.u, bt.v, bt.w, bt.op, prune_bounds=del_prune), f"batch {bi}")
        for _, g in reps:
            assert_edges_equal(g.sparsifier(), g1.sparsifier(), "H")
            assert_edges_equal(g.edges(), g1.edges(), "G")
            assert g.stats()["walked"] == g1.stats()["walked"] and g.stats()["steps"] == g1.stats()["steps"]
    assert_edges_equal(g1.sparsifier(), o.edges("H"), "oracle H")
    for ctx, _ in reps + [(ctx1, g1)]:
        ctx.close()


def test_sharded_power_law_with_hubs():
    """R-MAT scale 16: hubs, long-list fallbacks and isolated starts."""
    wl, st = W.make_rmat(16, 600_000)
    rng = np.random.default_rng(5)
    reps = _graphs(wl, 2)
    (ctx1, g1), = _graphs(wl, 1)
    for bi in range(2):
        bt = st.next_batch(6000, 4000)
        ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
        outs, _ = _sharded(reps, ups, rng)
        ref = g1.apply(ups)
        assert ref["fallback"].sum() > 0
        for r in outs:
            assert_same_outputs(r, ref)
        for _, g in reps:
            assert_edges_equal(g.sparsifier(), g1.sparsifier(), "H")
    for ctx, _ in reps + [(ctx1, g1)]:
        ctx.close()


def test_sharded_batch_rejects_incomplete_records_and_other_work():
    wl, st = W.make_grid(24, 24)
    reps = _graphs(wl, 2)
    bt = st.next_batch(100, 80)
    ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
    for r, (_, g) in enumerate(reps):
        g.shard_begin(ups, r, 2)
    recs = np.concatenate([g.shard_export() for _, g in reps])
    g0 = reps[0][1]
    with pytest.raises(D.DgError) as e:  # one walked update missing
        g0.shard_commit(recs[1:])
    assert e.value.code == -1
    with pytest.raises(D.DgError) as e:  # one walked update twice
        g0.shard_commit(np.concatenate([recs, recs[:1]]))
    assert e.value.code == -1
    with pytest.raises(D.DgError) as e:  # no other batch while the sharded one is open
        g0.apply(ups)
    assert e.value.code == -5
    with pytest.raises(D.DgError) as e:
        g0.shard_begin(ups, 2, 2)
    assert e.value.code in (-1, -5)
    (ctx1, g1), = _graphs(wl, 1)
    ref = g1.apply(ups)
    for _, g in reps:  # the complete records still commit
        assert_same_outputs(g.shard_commit(recs), ref)
        assert_edges_equal(g.sparsifier(), g1.sparsifier(), "H")
    for ctx, _ in reps + [(ctx1, g1)]:
        ctx.close()
