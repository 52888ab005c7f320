"""Failure detection without a GPU fault: the bounded device-side waits.

The finalizing warps of the batched walk wait for completed updates on a
queue, and every such wait gives up after a bounded number of polls, records
the failure in the batch's error word and lets the kernel return.  Here the
limit is set to zero polls, so the wait of a batch with walked updates must
give up: the call returns DG_E_TIMEOUT instead of hanging or trapping, the CUDA
context stays usable, and a fresh context then computes the next batch as the
oracle does.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import pair, step_both

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cuda_graphs", [True, False])
def test_finalize_wait_gives_up_with_timeout(cuda_graphs):
    import torch

    wl, st = W.make_grid(32, 32)
    bt = st.next_batch(150, 100)
    ctx = D.Context(cuda_graphs=cuda_graphs, autotune=False)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    ctx.debug_set_wait_limit(0)
    with pytest.raises(D.DgError) as e:
        g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    assert e.value.code == -4 and "gave up" in str(e.value)
    torch.cuda.synchronize()  # the device context survived
    g.unload()
    ctx.debug_set_wait_limit(-1)
    g2 = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)  # the same context, default limit again
    g2.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    res = g2.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
    assert (res["status"] == 0).all() and res["walked"].sum() > 0
    ctx.close()
    # a fresh context: the same batch and the next one match the oracle
    ctx, g, o = pair(wl.n, wl.a, wl.b, wl.w, wl.h_ids, ctx_kw=dict(cuda_graphs=cuda_graphs))
    step_both(g, o, bt.u, bt.v, bt.w, bt.op, where="after timeout")
    b2 = st.next_batch(120, 80)
    step_both(g, o, b2.u, b2.v, b2.w, b2.op, where="after timeout, next batch")
    ctx.close()
