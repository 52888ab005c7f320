"""dg_walk_estimate_noalloc: the walk estimate for callers that cannot allocate
device memory while they run (a stream capture in progress, a latency-critical
thread, an embedder whose device memory is already handed out).  Its scratch is
a fixed static device array inside the library.

The estimate it writes for an insertion query must equal what dg_apply_updates
reports for the same insertion walked on the same sparsifier (same update id,
endpoints and weight): hit, nhits, best walker and steps exactly, R~ to 0 ULP,
the tolerance every parity test here uses.  Checked on two calls in a row, the
second after the first batch changed H.  A deletion query walks the current G
unpruned, so on the G a deletion batch left behind it equals that batch's
walked deletions under del_prune = 0.  This file is collected last.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _queries(bt, first_id):
    q = np.zeros(len(bt), D.QUERY_DTYPE)
    q["u"], q["v"], q["w"] = bt.u, bt.v, bt.w
    q["kind"] = D.OP_INSERT
    q["id"] = first_id + np.arange(len(bt), dtype=np.uint64)
    return q


def test_noalloc_estimate_matches_apply_updates_twice():
    import torch

    wl, st = W.make_grid(48, 48)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    stream = torch.cuda.current_stream()
    for call in range(2):
        bt = st.next_batch(1500, 0)  # insertions of new edges only: the walks run on H itself
        q = _queries(bt, g.next_update_id)
        d_q = torch.from_numpy(q.view(np.uint8)).cuda()
        d_out = torch.full((len(q) * 32,), 0xAB, dtype=torch.uint8, device="cuda")
        g.walk_estimate_noalloc(d_q.data_ptr(), len(q), d_out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        est = d_out.cpu().numpy().view(D.ESTIMATE_DTYPE)
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        assert (res["status"] == 0).all() and (est["status"] == 0).all()
        for f in ("hit", "nhits", "best_walker", "steps"):
            assert np.array_equal(est[f].astype(np.int64), res[f].astype(np.int64)), (call, f)
        assert np.array_equal(est["r_est"].view(np.uint64), res["r_est"].view(np.uint64)), call
        assert est["hit"].sum() > 0 and (est["hit"] == 0).sum() > 0
    ctx.close()


def test_noalloc_deletion_queries_match_unpruned_deletions():
    import torch

    wl, st = W.make_grid(48, 48)
    ctx = D.Context(del_prune=False)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for call in range(2):
        bt = st.next_batch(0, 1200)  # deletions only: afterwards G is the batch's G_b
        q = _queries(bt, g.next_update_id)
        q["kind"] = D.OP_DELETE
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        d_q = torch.from_numpy(q.view(np.uint8)).cuda()
        d_out = torch.full((len(q) * 32,), 0xAB, dtype=torch.uint8, device="cuda")
        g.walk_estimate_noalloc(d_q.data_ptr(), len(q), d_out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        est = d_out.cpu().numpy().view(D.ESTIMATE_DTYPE)
        walked = res["walked"] == 1
        assert walked.sum() > 50 and (est["status"] == 0).all()
        for f in ("hit", "nhits", "best_walker", "steps"):
            assert np.array_equal(est[f][walked].astype(np.int64), res[f][walked].astype(np.int64)), (call, f)
        assert np.array_equal(est["r_est"][walked].view(np.uint64), res["r_est"][walked].view(np.uint64)), call
        assert est["hit"][walked].sum() > 0
    ctx.close()


def test_noalloc_ordered_against_the_next_batch():
    """The estimate is issued on a side stream and the batch that changes H
    follows at once on another stream, with no synchronization in between:
    the batch waits for the estimate's kernels, so the estimate still sees H
    before the batch."""
    import torch

    wl, st = W.make_grid(48, 48)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    side = torch.cuda.Stream()
    for call in range(2):
        bt = st.next_batch(3000, 0)
        q = _queries(bt, g.next_update_id)
        d_q = torch.from_numpy(q.view(np.uint8)).cuda()
        d_out = torch.empty(len(q) * 32, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        g.walk_estimate_noalloc(d_q.data_ptr(), len(q), d_out.data_ptr(), side.cuda_stream)
        res = g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
        side.synchronize()
        est = d_out.cpu().numpy().view(D.ESTIMATE_DTYPE)
        for f in ("hit", "nhits", "best_walker", "steps"):
            assert np.array_equal(est[f].astype(np.int64), res[f].astype(np.int64)), (call, f)
        assert np.array_equal(est["r_est"].view(np.uint64), res["r_est"].view(np.uint64)), call
    ctx.close()


def test_noalloc_rejects_oversize_without_device_work():
    ctx = D.Context()
    wl, _ = W.make_grid(8, 8)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    with pytest.raises(D.DgError) as e:
        g.walk_estimate_noalloc(0, D.NOALLOC_MAX_QUERIES + 1, 0)
    assert e.value.code == -1 and "DG_NOALLOC_MAX_QUERIES" in str(e.value)
    ctx.close()
    # within the query limit but over the walker limit (queries x s)
    ctx = D.Context(s=64)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    nq = D.NOALLOC_MAX_WALKERS // 64 + 1
    assert nq <= D.NOALLOC_MAX_QUERIES
    with pytest.raises(D.DgError) as e:
        g.walk_estimate_noalloc(0, nq, 0)
    assert e.value.code == -1 and "DG_NOALLOC_MAX_WALKERS" in str(e.value)
    # no queries: DG_OK and nothing launched
    before = ctx.launch_count()
    g.walk_estimate_noalloc(0, 0, 0)
    assert ctx.launch_count() == before
    ctx.close()
