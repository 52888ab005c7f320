"""GPU (CUDA library, through the C ABI) vs CPU oracle, element by element.

Everything integer (statuses, flags, hit counts, best walkers, step counts,
walk paths, edge sets) must match exactly; R~ and weights must match to 0 ULP
(both sides add r_e in walk order and round each FP64 operation on its own).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal, assert_results_equal, assert_same_outputs, pair, step_both
from tests.helpers import random_connected, ring

pytestmark = pytest.mark.gpu


def test_grid64_insertions_paths_and_records():
    """The 64x64 grid workload: 200 insertions <= 4 hops apart, s=32, T=100;
    walker paths, stop reasons and step counts agree walker by walker."""
    wl, st = W.make_grid(64, 64)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, ctx_kw=dict(record_walkers=True))
    bt = st.next_batch(200, 0)
    res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    ref = o.apply(bt.u, bt.v, bt.w, bt.op, walkers=True, paths=True)
    assert_results_equal(res, ref, "grid64")
    rec = g.walker_records(len(bt))
    assert np.array_equal(rec["reason"], ref["walkers"]["reason"])
    assert np.array_equal(rec["steps"], ref["walkers"]["steps"])
    # every walker's path row: the vertices up to its (cut) step count, then -1
    assert np.array_equal(rec["paths"], ref["paths"])
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    assert res["accepted"].sum() > 0 and res["hit"].sum() > 0
    ctx.close()


def test_grid64_step_limit_10():
    wl, st = W.make_grid(64, 64, T=10)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, T=10)
    bt = st.next_batch(200, 0)
    step_both(g, o, bt.u, bt.v, bt.w, bt.op, where="grid64 T=10")
    ctx.close()


@pytest.mark.parametrize("early_exit,del_prune", [(True, True), (False, False), (True, False)])
def test_grid_mixed_stream(early_exit, del_prune):
    """Several fully dynamic batches (insertions and deletions interleaved)."""
    wl, st = W.make_grid(32, 32)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, early_exit=early_exit, ctx_kw=dict(del_prune=del_prune))
    for b in range(4):
        bt = st.next_batch(150, 150)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"batch {b}")
    ctx.close()


@pytest.mark.parametrize("K", [0.0, 4.0, 7.5, 1e300, math.inf])
def test_threshold_ties_and_extremes(K):
    """Unit weights make w_pq * R land exactly on K (a hit, reading R4); K = 0
    and K = +inf are the ends of the threshold range.  The kernel's integer
    form of the threshold test must decide every step as the product does."""
    rng = np.random.default_rng(11)
    n = 200
    a, b, w = random_connected(n, 300, rng, unit=True)
    h = W.init_sparsifier(n, a, b, w, rng, frac=0.2)
    ctx, g, o = pair(n, a, b, w, h, K=K, T=40, s=16)
    wl = W.Workload("unit", n, *W.canonical(a, b, w), h_ids=h)
    stream = W.UpdateStream(wl, rng, ("uniform",), lambda r, u, v: r.choice([0.5, 1.0, 2.0], len(u)))
    for bi in range(3):
        bt = stream.next_batch(150, 30)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"K={K} batch {bi}")
    ctx.close()


@pytest.mark.parametrize("s,T,K", [(1, 1, 100.0), (1, 40, 3.0), (33, 2, 100.0), (64, 15, 8.0), (7, 17, 0.0)])
def test_degenerate_walk_parameters(s, T, K):
    """One walker per update, a one-step limit, updates whose walkers span more
    than one warp, step limits just below and above the resume-point spacing,
    K = 0; a graph with isolated vertices so some walks start at degree 0."""
    rng = np.random.default_rng(300 + s + T)
    n = 150
    a, b, w = random_connected(n - 20, 220, rng, 0.2, 5.0)  # vertices n-20..n-1 stay isolated at first
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, s=s, T=T, K=K, ctx_kw=dict(record_walkers=True))
    ups = _mixed_updates(rng, n, a, b, 160)
    ups += [(n - 1, int(rng.integers(0, n - 20)), 1.0, 0), (n - 2, n - 3, 2.0, 0)]  # walks from isolated starts
    cols = list(zip(*ups))
    res, ref = step_both(g, o, list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), where=f"s={s} T={T}")
    assert (res["walked"] == 1).any()
    for k in range(3):  # further batches on the evolved graphs
        ups = _mixed_updates(rng, n, *[np.array(x) for x in zip(*sorted(o_edges(o)))], 120)
        cols = list(zip(*ups))
        step_both(g, o, list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), where=f"s={s} T={T} b{k}")
    ctx.close()


def test_long_step_limit_resume_points():
    """With a step limit this long the deletion walkers' step records would
    not fit their memory budget, so the argmin path is replayed from resume
    points (every 4096 steps here) instead: results, H and G equal the oracle."""
    rng = np.random.default_rng(77)
    n = 120
    a, b, w = random_connected(n, 200, rng, 0.2, 5.0)
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, s=32, T=20000, K=50.0)
    for k in range(2):
        ups = _mixed_updates(rng, n, *[np.array(x) for x in zip(*sorted(o_edges(o)))], 60)
        cols = list(zip(*ups))
        res, _ = step_both(g, o, list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), where=f"long T b{k}")
        assert (res["walked"] == 1).any()
    ctx.close()


def test_empty_and_all_invalid_batches():
    wl, st = W.make_grid(16, 16)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    before = g.sparsifier()
    res = g.apply(D.make_updates([], [], [], []))
    assert len(res) == 0 and g.next_update_id == 0
    bad = [(3, 3, 1.0, 0), (wl.n, 1, 1.0, 0), (1, 2, -2.0, 0), (1, 2, 1.0, 7), (0, 5, 0.0, 1)]
    cols = list(zip(*bad))
    res, _ = step_both(g, o, list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), where="all invalid")
    assert (res["status"] != 0).all() and (res["walked"] == 0).all()
    assert_edges_equal(g.sparsifier(), before, "H unchanged")
    assert g.next_update_id == len(bad)  # invalid updates still consume ids
    ctx.close()


def o_edges(o):
    a, b, _ = o.edges("G")
    return list(zip(a.tolist(), b.tolist()))


def _mixed_updates(rng, n, a, b, count):
    """Insertions between random pairs and deletions of existing edges (some
    repeated or invalid), as (u, v, w, op) tuples."""
    cur = list(zip(np.asarray(a).tolist(), np.asarray(b).tolist()))
    ups = []
    for _ in range(count):
        r = rng.random()
        if r < 0.5:
            x, y = (int(t) for t in rng.integers(0, n, 2))
            ups.append((x, y, float(rng.uniform(0.2, 5.0)), 0))
        elif r < 0.95 and cur:
            x, y = cur[int(rng.integers(0, len(cur)))]
            ups.append((y, x, 0.0, 1) if rng.random() < 0.5 else (x, y, 0.0, 1))
        else:
            ups.append((int(rng.integers(0, n)), int(rng.integers(0, n)), 0.0, 1))
    return ups


def test_deletion_pruning_walker_records():
    """Pruned deletion walkers (the default): every walker's stop reason and
    step count equal the oracle's under the exact rule (a walker of a deletion
    with a hit stops at its first step whose resistance exceeds R~), and its
    recorded path equals the oracle's walk cut there, -1 padded; the pruned
    steps are far fewer than the unpruned ones."""
    wl, st = W.make_grid(48, 48)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, ctx_kw=dict(record_walkers=True))
    skipped = 0
    for b in range(2):
        bt = st.next_batch(100, 400)
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        ref = o.apply(bt.u, bt.v, bt.w, bt.op, walkers=True, paths=True, prune_bounds=True)
        assert_results_equal(res, ref, f"pruned batch {b}")
        assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
        rec = g.walker_records(len(bt))
        lo = ref["walkers_lo"]
        assert np.array_equal(rec["reason"], lo["reason"]), b
        assert np.array_equal(rec["steps"], lo["steps"]), b
        expect = ref["paths"].copy()
        for i in range(len(bt)):
            for k in range(wl.s):
                expect[i, k, lo["steps"][i, k] + 1:] = -1
        assert np.array_equal(rec["paths"], expect), b
        dels = np.nonzero((bt.op == 1) & (res["walked"] == 1))[0]
        assert (rec["reason"][dels] == 5).any() and res["hit"][dels].sum() > 0
        skipped += int((ref["steps"][dels] - res["steps"][dels]).sum())
    assert skipped > 0
    ctx.close()


def test_invalid_and_repeated_updates():
    """Statuses of invalid updates and the batch-local view of repeated edges."""
    rng = np.random.default_rng(1)
    n = 40
    a, b, w = random_connected(n, 40, rng)
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, T=20, s=8, K=12.0)
    x, y = int(a[h][0]), int(b[h][0])
    nx, ny = 0, 0
    present = set(zip(a.tolist(), b.tolist()))
    for p in range(n):
        for q in range(p + 1, n):
            if (p, q) not in present:
                nx, ny = p, q
                break
        if nx != ny:
            break
    ups = [
        (x, y, 0.0, 1), (y, x, 2.5, 0), (x, y, 0.0, 1), (x, y, 3.5, 0),  # delete/insert/delete/insert one H edge
        (nx, ny, 1.5, 0), (ny, nx, 0.0, 1),                               # insert then delete a new edge
        (nx, ny, 1.0, 1),                                                 # delete of an absent edge
        (3, 3, 1.0, 0), (n + 5, 1, 1.0, 0), (-1, 2, 1.0, 1),             # self-loop, bad vertices
        (1, 2, -1.0, 0), (1, 2, float("nan"), 0), (1, 2, float("inf"), 0), (1, 2, 1.0, 9),
        (int(a[0]), int(b[0]), 1.0, 0),                                    # duplicate insert
    ]
    cols = list(zip(*ups))
    res, ref = step_both(g, o, list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), where="invalid")
    assert set(res["status"].tolist()) >= {0, 1, 2, 3, 4, 5, 6}
    ctx.close()


def test_ring_recovery_and_fallback():
    n = 9
    a, b, w = ring(n)
    keep = np.nonzero(~((a == 2) & (b == 3)))[0]
    for T, want_fallback in ((n - 1, 0), (3, 1)):
        ctx, g, o = pair(n, a, b, w, keep, T=T, s=8)
        res, _ = step_both(g, o, [0], [1], [0.0], [1], where=f"ring T={T}")
        assert res["fallback"][0] == want_fallback
        ctx.close()


def _hub_graph(rng, n, hub_deg, h_frac):
    """A ring over vertices 3..n-1, hubs 0, 1, 2 joined to each other and to
    hub_deg[h] random ring vertices; H(0) = the ring, the hub triangle and a
    fraction h_frac of every hub's other edges."""
    edges = {}
    for i in range(3, n):
        j = 3 + (i - 3 + 1) % (n - 3)
        edges[(min(i, j), max(i, j))] = True
    for h, d in enumerate(hub_deg):
        for y in rng.choice(np.arange(3, n), d, replace=False):
            edges[(h, int(y))] = rng.random() < h_frac
    for e in ((0, 1), (0, 2), (1, 2)):
        edges[e] = True
    keys = sorted(edges)
    a = np.array([k[0] for k in keys], np.int32)
    b = np.array([k[1] for k in keys], np.int32)
    in_h = np.array([edges[k] for k in keys])
    return a, b, in_h


@pytest.mark.parametrize("walk_mode", ["batched", "per_update"])
def test_long_list_fallback_split_scan(walk_mode):
    """Fallback (no walker reached v; minimum-resistance G_b edge not in H' at
    each endpoint) at endpoints with 1.5k to 7k neighbours: the CUDA path
    splits such lists into chunks of 2048 entries scanned by separate blocks
    and claims each endpoint once per batch.  Many deletions share a hub, one
    joins two hubs; a few hub edges outside H share the top weight, in
    different chunks, so the smaller neighbour id breaks the tie across
    chunks.  Two batches: the second picks the next minima after the first
    batch's recovered edges joined H, and must not see the first batch's
    claims.  A step limit of 2 makes most deletions fall back."""
    rng = np.random.default_rng(77)
    n = 9000
    a, b, in_h = _hub_graph(rng, n, (7000, 4500, 1500), 0.3)
    w = rng.uniform(0.1, 10.0, a.size)
    for h in range(3):  # tied top weights outside H, spread over the list
        idx = np.nonzero((a == h) & (b >= 3) & ~in_h)[0]
        w[rng.choice(idx, 4, replace=False)] = 20.0
    ctx, g, o = pair(n, a, b, w, np.nonzero(in_h)[0], seed=5, K=100.0, T=2, s=4,
                     ctx_kw=dict(walk_mode=walk_mode, cuda_graphs=walk_mode == "batched"))
    hub_h = np.nonzero(in_h & (a <= 2) & (b >= 3))[0]
    picks = rng.permutation(hub_h)
    plans = [picks[:260], picks[260:480]]
    for bi, ids in enumerate(plans):
        u, v = a[ids].copy(), b[ids].copy()
        flip = rng.random(ids.size) < 0.5  # either endpoint first
        u[flip], v[flip] = v[flip], u[flip]
        u = np.append(u, [0, 1][bi])
        v = np.append(v, [1, 2][bi])  # a deletion between two hubs
        res, _ = step_both(g, o, u, v, np.zeros(u.size), np.ones(u.size, np.int32),
                           where=f"{walk_mode} batch {bi}")
        assert res["fallback"].sum() > 0.5 * u.size
        assert res["nrecovered"].sum() > 0
    ctx.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_graphs_many_batches(seed):
    rng = np.random.default_rng(100 + seed)
    n = 300
    a, b, w = random_connected(n, 700, rng, 0.1, 10.0)
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, seed=seed * 7 + 3, K=[5.0, 50.0, 500.0][seed], T=[30, 100, 60][seed],
                     s=[32, 16, 48][seed])
    wl = W.Workload("rand", n, *W.canonical(a, b, w), h_ids=h)
    stream = W.UpdateStream(wl, rng, ("uniform",), lambda r, u, v: r.uniform(0.1, 10.0, len(u)))
    for bi in range(5):
        bt = stream.next_batch(int(rng.integers(1, 120)), int(rng.integers(0, 120)))
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"seed {seed} batch {bi}")
    ctx.close()


@pytest.mark.parametrize("del_prune", [False, True])
def test_execution_forms_agree(del_prune):
    """Per-update launches, CUDA-graph replay, eager batched and every walk
    launch shape (threads per block, walkers per thread, lanes per walker,
    frontier tile) give bit-identical outputs, with and without deletion
    pruning."""
    wl, st = W.make_grid(40, 40)
    batches = [st.next_batch(300, 200) for _ in range(3)]
    outs = []
    configs = [dict(walk_mode="batched", cuda_graphs=True), dict(walk_mode="batched", cuda_graphs=False),
               dict(walk_mode="per_update", cuda_graphs=False)]
    for kw in configs:
        ctx = D.Context(del_prune=del_prune, **kw)
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        rs = [g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op)) for bt in batches]
        outs.append((rs, g.sparsifier()))
        ctx.close()
    for shape in [(32, 1, 0), (64, 2, 4), (256, 4, 0), (128, 2, 1)]:
        ctx = D.Context(del_prune=del_prune)
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        g.set_walk_shape(*shape)
        rs = [g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op)) for bt in batches]
        outs.append((rs, g.sparsifier()))
        ctx.close()
    # lanes per walker and the frontier tile (the tiled launch)
    for lanes, tile, block in [(1, 1, 256), (2, 4, 128), (4, 16, 256), (8, 1, 64), (32, 3, 256), (32, 1, 32)]:
        ctx = D.Context(del_prune=del_prune)
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        g.set_walk_shape(block, 1, 0)
        g.set_walk_coop(lanes, tile)
        rs = [g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op)) for bt in batches]
        st_ = g.stats()
        assert (st_["walk_lanes"], st_["walk_tile"]) == (lanes, tile)
        outs.append((rs, g.sparsifier()))
        ctx.close()
    ref_rs, ref_h = outs[0]
    for rs, hh in outs[1:]:
        for r0, r1 in zip(ref_rs, rs):
            assert_same_outputs(r0, r1)
        assert_edges_equal(hh, ref_h, "H")


def test_device_io_matches_host_io():
    import torch
    wl, st = W.make_grid(32, 32)
    bt = st.next_batch(200, 100)
    ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
    out = []
    for mode in ("host", "pinned", "device"):
        ctx = D.Context()
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        if mode == "device":
            d_ups = torch.from_numpy(ups.view(np.uint8)).cuda()
            d_res = torch.zeros(len(ups) * 32, dtype=torch.uint8, device="cuda")
            g.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            res = d_res.cpu().numpy().view(D.RESULT_DTYPE)
        elif mode == "pinned":  # pinned host arrays are copied without staging
            p_ups = torch.empty(len(ups) * 24, dtype=torch.uint8, pin_memory=True).numpy().view(D.UPDATE_DTYPE)
            p_res = torch.empty(len(ups) * 32, dtype=torch.uint8, pin_memory=True).numpy().view(D.RESULT_DTYPE)
            p_ups[:] = ups
            res = g.apply(p_ups, out=p_res)
        else:
            res = g.apply(ups)
        out.append((res.copy(), g.sparsifier()))
        ctx.close()
    for k in (1, 2):
        assert_same_outputs(out[0][0], out[k][0])
        assert_edges_equal(out[0][1], out[k][1], "H")


def test_pool_growth_and_compaction_keep_results():
    """No slack and no headroom force relocations, pool growth and retries."""
    wl, st = W.make_grid(24, 24)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, ctx_kw=dict(slack=1.0, overflow=0.0))
    for bi in range(4):
        bt = st.next_batch(400, 50)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"tight batch {bi}")
    g.compact()
    bt = st.next_batch(100, 100)
    step_both(g, o, bt.u, bt.v, bt.w, bt.op, where="after compaction")
    ctx.close()


def test_checkpoint_resume_by_update_id():
    """Restoring H, G and the update sequence number replays bit-identically."""
    wl, st = W.make_grid(24, 24)
    b1 = st.next_batch(100, 60)
    b2 = st.next_batch(100, 60)
    ctx, g, _ = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    g.apply(D.make_updates(b1.u, b1.v, b1.w, b1.op))
    ga, gb, gw = g.edges()
    ha, hb, _ = g.sparsifier()
    nid = g.next_update_id
    r_direct = g.apply(D.make_updates(b2.u, b2.v, b2.w, b2.op))
    g2 = ctx.load_graph(wl.n, ga, gb, gw)
    g2.init_sparsifier(ha, hb)
    g2.next_update_id = nid
    r_resumed = g2.apply(D.make_updates(b2.u, b2.v, b2.w, b2.op))
    assert_same_outputs(r_direct, r_resumed)
    assert_edges_equal(g.sparsifier(), g2.sparsifier(), "H")
    ctx.close()


def test_invalid_graph_inputs():
    ctx = D.Context()
    with pytest.raises(D.DgError) as e:
        ctx.load_graph(4, [0, 1], [1, 0], [1.0, 1.0])  # same edge twice
    assert e.value.code == -1
    with pytest.raises(D.DgError):
        ctx.load_graph(4, [0], [4], [1.0])  # vertex out of range
    with pytest.raises(D.DgError):
        ctx.load_graph(4, [0], [1], [0.0])  # weight not > 0
    g = ctx.load_graph(4, [0, 1], [1, 2], [1.0, 2.0])
    with pytest.raises(D.DgError):
        g.init_sparsifier([0], [2])  # not an edge of G
    g.init_sparsifier([0, 1, 0], [1, 2, 1])  # repeated pair kept once
    a, b, w = g.sparsifier()
    assert a.tolist() == [0, 1] and b.tolist() == [1, 2] and w.tolist() == [1.0, 2.0]
    ctx.close()


def test_invariants_subgraph_and_components():
    from oracle import checks
    wl, st = W.make_grid(32, 32)
    ctx, g, _ = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    for _ in range(3):
        bt = st.next_batch(200, 100)
        g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        ga, gb, gw = g.edges()
        ha, hb, hw = g.sparsifier()
        gm = dict(zip(zip(ga.tolist(), gb.tolist()), gw.tolist()))
        assert all(gm.get((x, y)) == ww for x, y, ww in zip(ha.tolist(), hb.tolist(), hw.tolist()))
        assert checks.n_components(wl.n, ha, hb) == checks.n_components(wl.n, ga, gb)
    ctx.close()


# the CUDA path's hub thresholds: a vertex becomes a hub at degree 32 and
# stays one down to 24 (a layout choice: entries pointing at it hold no cache)
HUB_HI, HUB_LO = 32, 24


def test_hub_references_and_status_flips():
    """Vertices of degree >= HUB_HI are referenced without cached list data (a
    layout choice of the CUDA path).  Walks through such hubs, changes of their
    lists, and hubs crossing the thresholds (down below HUB_LO, back up through
    HUB_HI) must leave every result, H and G equal to the oracle."""
    rng = np.random.default_rng(21)
    n = 4000
    edges = set()
    for hub, d in ((0, HUB_HI + 10), (1, HUB_HI + 2), (2, HUB_HI - 8)):
        for y in rng.choice(np.arange(3, n), d, replace=False):
            edges.add((hub, int(y)))
    perm = rng.permutation(n)
    for i in range(1, n):  # a random spanning tree keeps the graph connected
        x, y = int(perm[i]), int(perm[rng.integers(0, i)])
        edges.add((min(x, y), max(x, y)))
    while len(edges) < 9000:
        x, y = (int(t) for t in rng.integers(3, n, 2))
        if x != y:
            edges.add((min(x, y), max(x, y)))
    e = sorted(edges)
    a = np.array([p for p, _ in e], np.int32)
    b = np.array([q for _, q in e], np.int32)
    w = rng.uniform(0.5, 5.0, len(e))
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, T=60, s=16, K=40.0, ctx_kw=dict(record_walkers=True))
    cur = set(edges)

    def nbrs(x):
        return sorted(y for (p, q) in cur for y in ((q,) if p == x else (p,) if q == x else ()))

    def batch(dels, ins, extra=150):
        us, vs, ws, ops = [], [], [], []
        for x, y in dels:
            us.append(x); vs.append(y); ws.append(0.0); ops.append(1)
            cur.discard((min(x, y), max(x, y)))
        for x, y in ins:
            us.append(x); vs.append(y); ws.append(float(rng.uniform(0.5, 5.0))); ops.append(0)
            cur.add((min(x, y), max(x, y)))
        for _ in range(extra):  # random insertions elsewhere, walks start at random vertices
            x, y = (int(t) for t in rng.integers(3, n, 2))
            if x != y and (min(x, y), max(x, y)) not in cur:
                us.append(x); vs.append(y); ws.append(float(rng.uniform(0.5, 5.0))); ops.append(0)
                cur.add((min(x, y), max(x, y)))
        order = rng.permutation(len(us))
        return ([us[i] for i in order], [vs[i] for i in order], [ws[i] for i in order], [ops[i] for i in order])

    def new_nbrs(x, k):
        have = set(nbrs(x))
        cand = [y for y in range(3, n) if y != x and y not in have]
        return [(x, int(y)) for y in rng.choice(cand, k, replace=False)]

    d0 = len(nbrs(0))
    assert d0 >= HUB_HI and len(nbrs(1)) >= HUB_HI and len(nbrs(2)) < HUB_HI
    plans = [  # hub 0 drops to HUB_LO (stays a hub), vertex 2 rises past HUB_HI (joins)
        (lambda: [(0, y) for y in nbrs(0)[: d0 - HUB_LO]], lambda: new_nbrs(2, 12)),
        (lambda: [(0, y) for y in nbrs(0)[:3]], lambda: new_nbrs(1, 5)),      # hub 0 below HUB_LO (leaves)
        (lambda: [(1, y) for y in nbrs(1)[:4]], lambda: new_nbrs(0, 20)),     # hub 0 back above HUB_HI (joins again)
    ]
    for bi, (dl, il) in enumerate(plans):
        u, v, ww, op = batch(dl(), il())
        step_both(g, o, u, v, ww, op, where=f"hub batch {bi}")
    ctx.close()


def test_power_law_hubs_many_batches():
    """A small symmetrised R-MAT graph has many hubs, most of which stay hubs
    from batch to batch while their neighbours' lists change: the cache refresh
    then visits only a stable hub's new entries and refreshes the others from
    the neighbour's side.  Walks through those hubs, the results, H and G must
    equal the oracle over several batches of insertions and deletions."""
    rng = np.random.default_rng(5)
    n, a, b = W.rmat(11, 12000, rng)
    w = rng.uniform(0.5, 5.0, len(a))
    h = W.init_sparsifier(n, a, b, w, rng)
    deg = np.bincount(np.concatenate([a, b]), minlength=n)
    assert (deg >= HUB_HI).sum() >= 20
    ctx, g, o = pair(n, a, b, w, h, T=40, s=16, K=60.0)
    wl = W.Workload("rmat_s11", n, a, b, w, h, K=60.0, T=40, s=16, seed=0)
    stream = W.UpdateStream(wl, rng, ("uniform",), lambda r, u, v: r.uniform(0.5, 5.0, len(u)))
    for bi in range(4):
        bt = stream.next_batch(300, 400)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"rmat batch {bi}")
    ctx.close()


def test_walk_refill_threshold():
    """The refill threshold changes only when warps start new walkers: every
    value gives the same outputs; values outside 1..32 are rejected."""
    wl, st = W.make_grid(40, 40)
    batches = [st.next_batch(300, 200) for _ in range(3)]
    outs = []
    for refill in (1, 7, 16, 32):
        ctx = D.Context(del_prune=False)
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        g.set_walk_shape(128, 1, 0, refill=refill)
        rs = [g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op)) for bt in batches]
        assert g.stats()["walk_refill"] == refill
        outs.append((rs, g.sparsifier()))
        for bad in (-1, 33):
            with pytest.raises(D.DgError):
                g.set_walk_shape(refill=bad)
        ctx.close()
    for rs, hh in outs[1:]:
        for r0, r1 in zip(outs[0][0], rs):
            assert_same_outputs(r0, r1)
        assert_edges_equal(hh, outs[0][1], "H")


def test_mesh3d_small_multi_batch():
    wl, st = W.make_mesh3d(24, 24, 24)
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    for bi in range(3):
        bt = st.next_batch(2000, 2000)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"mesh24 batch {bi}")
    ctx.close()


def test_mesh3d_full_size_batch():
    """The 100x100x100 mesh (1M vertices, 2.97M edges) at its full batch size
    (10k insertions + 10k deletions), in the launch form the benchmark times
    (batched, CUDA graph): every update result and the final H, G match."""
    wl, st = W.make_mesh3d()
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
    for bi in range(2):
        bt = st.next_batch(10000, 10000)
        res, ref = step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"mesh100 batch {bi}")
        assert (res["status"] == 0).all()
    assert g.stats()["graph_replayed"] == 1
    ctx.close()


def test_set_walk_coop_rejects_bad_values():
    wl, _ = W.make_grid(8, 8)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    for lanes, tile in [(3, 0), (0, 0), (64, 1), (1, -1), (1, 17)]:
        with pytest.raises(D.DgError) as e:
            g.set_walk_coop(lanes, tile)
        assert e.value.code == -1
    ctx.close()


def test_autotuner_tries_every_work_shape():
    """The first large batch runs the autotuner: its trial log covers the
    threads-per-block / walkers-per-thread shapes, the refill thresholds and
    the tiled launch's lanes per walker and tiles, and the batch's outputs
    equal those of a fixed shape."""
    wl, st = W.make_mesh3d(24, 24, 24, seed=3)
    bt = st.next_batch(3000, 2000)
    outs = []
    for tune in (True, False):
        ctx = D.Context()
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        if not tune:
            g.set_walk_shape(256, 1, 0)
        outs.append(g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op)))
        if tune:
            assert g.stats()["autotuned"] == 1
            log = g.tune_log()
            shapes = {(d["lanes"], d["tile"]) for d, _ in log}
            assert {(1, 0), (2, 1), (4, 1), (8, 1), (32, 1), (32, 4), (1, 4)} <= shapes
            assert {d["refill"] for d, _ in log} >= {1, 8, 16, 24, 32}
            assert all(ms > 0 for _, ms in log)
        ctx.close()
    assert_same_outputs(outs[0], outs[1])


def test_work_shapes_agree_on_a_power_law_graph():
    """Hubs (HUBREF entries, slot hints) under every work shape: the tiled
    launch's lanes per walker and tiles give the outputs of the persistent
    launch, byte for byte, and both match the oracle."""
    wl, st = W.make_rmat(14, 150_000, seed=9)
    batches = [st.next_batch(1500, 1000) for _ in range(2)]
    outs = []
    for lanes, tile, block in [(1, 0, 256), (1, 4, 256), (4, 1, 128), (32, 2, 256)]:
        ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids)
        g.set_walk_shape(block, 1, 0)
        g.set_walk_coop(lanes, tile)
        rs = []
        for bt in batches:
            res, _ = step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"lanes {lanes} tile {tile}")
            rs.append(res)
        outs.append(rs)
        o.close()
        ctx.close()
    for rs in outs[1:]:
        for r0, r1 in zip(outs[0], rs):
            assert_same_outputs(r0, r1)


def test_merge_size_is_the_touched_lists():
    """The batch statistics report the size of G's list merge: every entry of
    a touched list read once (old list) and written once (new list).  The
    count equals the degrees of the vertices whose lists change, from the
    exported G before and after each batch, and the merge is timed."""
    rng = np.random.default_rng(11)
    n, a, b = W.rmat(11, 12000, rng)
    w = rng.uniform(0.5, 5.0, len(a))
    h = W.init_sparsifier(n, a, b, w, rng)
    ctx, g, o = pair(n, a, b, w, h, T=40, s=16, K=60.0)
    wl = W.Workload("rmat_s11", n, a, b, w, h, K=60.0, T=40, s=16, seed=0)
    stream = W.UpdateStream(wl, rng, ("uniform",), lambda r, u, v: r.uniform(0.5, 5.0, len(u)))

    def snapshot():
        ga, gb, _ = g.edges()
        deg = np.bincount(np.concatenate([ga, gb]), minlength=n)
        keys = set(zip(np.minimum(ga, gb).tolist(), np.maximum(ga, gb).tolist()))
        return deg, keys

    for bi in range(3):
        bt = stream.next_batch(300, 400)
        deg0, e0 = snapshot()
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        deg1, e1 = snapshot()
        st_ = g.stats()
        touched = set()
        for i in np.flatnonzero(res["status"] == 0):
            p = (int(min(bt.u[i], bt.v[i])), int(max(bt.u[i], bt.v[i])))
            if p in e0 or p in e1:  # absent before and after: no change record
                touched.update(p)
        t = np.fromiter(touched, np.int64)
        expect = int(deg0[t].sum() + deg1[t].sum())
        assert st_["merge_entries"] == expect, (bi, st_["merge_entries"], expect)
        assert st_["merge_ms"] > 0.0
        # the edge counts of the statistics are those of the current G and H
        assert st_["g_edges"] == len(e1)
        assert st_["h_edges"] == len(g.sparsifier()[0])
        assert_results_equal(res, o.apply(bt.u, bt.v, bt.w, bt.op, prune_bounds=g.ctx.del_prune), f"batch {bi}")
    ctx.close()
