"""GRASS-like initial sparsifier on the device (Section III-A; reading R20):
the given spanning forest plus the off-tree edges of largest stretch
w_e * R_F(e).  Every edge's stretch must equal the oracle's bit for bit
(root distances, lowest common ancestors and the stretch formula in the same
order), and the sparsifier must be the oracle's selection edge for edge."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import OracleGraph, grass_sparsifier, tree_stretch
from paper_2505_02741_b300 import dygrass as D
from paper_2505_02741_b300 import workloads as W
from tests.gpu_util import assert_edges_equal, step_both
from tests.helpers import random_connected

pytestmark = pytest.mark.gpu


def _check(n, a, b, w, tree, n_off):
    ctx = D.Context()
    g = ctx.load_graph(n, a, b, w)
    st = g.init_sparsifier_grass(a[tree], b[tree], n_off, with_stretch=True)
    ref = tree_stretch(n, a, b, w, tree)
    bad = np.nonzero(st.view(np.uint64) != ref.view(np.uint64))[0]
    assert bad.size == 0, (f"{bad.size} stretches differ, first at {bad[:5].tolist()}: gpu {st[bad[:5]].tolist()} "
                           f"oracle {ref[bad[:5]].tolist()} edges {list(zip(a[bad[:5]].tolist(), b[bad[:5]].tolist()))}")
    ids = grass_sparsifier(n, a, b, w, tree, n_off)
    ha, hb, hw = g.sparsifier()
    assert np.array_equal(ha, a[ids]) and np.array_equal(hb, b[ids])
    assert np.array_equal(hw.view(np.uint64), w[ids].view(np.uint64))
    return ctx, g, ids


@pytest.mark.parametrize("name", ["grid", "mesh", "rmat", "random"])
def test_grass_init_matches_oracle(name):
    if name == "grid":
        wl, _ = W.make_grid(40, 40)
    elif name == "mesh":
        wl, _ = W.make_mesh3d(12, 12, 12)
    elif name == "rmat":
        wl, _ = W.make_rmat(14, 120_000)  # hubs, isolated vertices, many trees
    else:
        rng = np.random.default_rng(3)
        n = 500
        a, b, w = random_connected(n, 1500, rng, 0.1, 9.0)
        wl = W.Workload("random", n, a, b, w, np.zeros(0, np.int64))
    tree = W.spanning_forest(wl.n, wl.a, wl.b, wl.w)
    n_off = (wl.m - tree.size) // 10
    ctx, g, _ = _check(wl.n, wl.a, wl.b, wl.w, tree, n_off)
    ctx.close()


def test_grass_forest_that_does_not_span():
    """Dropping forest edges splits trees: the edges between them have
    infinite stretch and are taken first."""
    wl, _ = W.make_grid(24, 24)
    tree = W.spanning_forest(wl.n, wl.a, wl.b, wl.w)
    part = tree[::3]
    ctx, g, ids = _check(wl.n, wl.a, wl.b, wl.w, part, 50)
    st = tree_stretch(wl.n, wl.a, wl.b, wl.w, part)
    assert np.isinf(st[ids[~np.isin(ids, part)]]).all()
    ctx.close()


def test_grass_rejects_cycles_and_non_edges():
    wl, _ = W.make_grid(16, 16)
    ctx = D.Context()
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    tree = W.spanning_forest(wl.n, wl.a, wl.b, wl.w)
    off = np.setdiff1d(np.arange(wl.m), tree)
    cyc = np.concatenate([tree, off[:1]])  # n edges on n vertices: a cycle
    with pytest.raises(D.DgError) as e:
        g.init_sparsifier_grass(wl.a[cyc], wl.b[cyc], 10)
    assert e.value.code == -1
    with pytest.raises(D.DgError) as e:
        g.init_sparsifier_grass(np.array([0], np.int32), np.array([wl.n - 1], np.int32), 10)
    assert e.value.code == -1
    ctx.close()


def test_batches_on_grass_sparsifier_match_oracle():
    """The update stream runs on the GRASS-like H(0) as on any other."""
    wl, st = W.make_mesh3d(14, 14, 14)
    tree = W.spanning_forest(wl.n, wl.a, wl.b, wl.w)
    n_off = (wl.m - tree.size) // 10
    ctx, g, ids = _check(wl.n, wl.a, wl.b, wl.w, tree, n_off)
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w)
    o.init_sparsifier(wl.a[ids], wl.b[ids])
    for bi in range(3):
        bt = st.next_batch(400, 400)
        step_both(g, o, bt.u, bt.v, bt.w, bt.op, where=f"grass batch {bi}")
    assert_edges_equal(g.sparsifier(), o.edges("H"), "H")
    ctx.close()
