"""Shared helpers of the GPU parity tests: run the same seeded input through the
CUDA library and through the CPU oracle and compare element by element."""
from __future__ import annotations

import numpy as np

from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D

FIELDS = ("status", "walked", "hit", "accepted", "fallback", "nhits", "best_walker", "nrecovered", "steps")


def assert_results_equal(gpu: np.ndarray, orc: dict, where=""):
    """Exact comparison.  When the oracle ran with prune_bounds (the GPU prunes
    deletion walkers), nhits and steps are compared with the oracle's counts
    under the exact pruning rule (every walker of a deletion with a hit stops
    at its first step whose resistance exceeds R~)."""
    pruned = "nhits_min" in orc
    for f in FIELDS:
        g = np.asarray(gpu[f]).astype(np.int64)
        src = {"nhits": "nhits_min", "steps": "steps_lo"}.get(f, f) if pruned else f
        o = np.asarray(orc[src]).astype(np.int64)
        if not np.array_equal(g, o):
            bad = np.nonzero(g != o)[0][:10]
            raise AssertionError(f"{where} field {f} differs at {bad.tolist()}: gpu {g[bad].tolist()} "
                                 f"oracle {o[bad].tolist()}")
    # R~ is compared bit for bit (0 ULP), +inf included
    gb = np.asarray(gpu["r_est"], np.float64).view(np.uint64)
    ob = np.asarray(orc["r_est"], np.float64).view(np.uint64)
    if not np.array_equal(gb, ob):
        bad = np.nonzero(gb != ob)[0][:10]
        raise AssertionError(f"{where} r_est differs at {bad.tolist()}: gpu {gpu['r_est'][bad].tolist()} "
                             f"oracle {np.asarray(orc['r_est'])[bad].tolist()}")


def assert_edges_equal(gpu_edges, orc_edges, what):
    ga, gb, gw = gpu_edges
    oa, ob, ow = orc_edges
    assert ga.size == oa.size, f"{what}: {ga.size} edges on the GPU, {oa.size} in the oracle"
    assert np.array_equal(ga, oa) and np.array_equal(gb, ob), f"{what}: edge sets differ"
    assert np.array_equal(gw.view(np.uint64), ow.view(np.uint64)), f"{what}: weights differ"


def assert_same_outputs(r0: np.ndarray, r1: np.ndarray):
    """Two GPU result arrays of the same batch: every byte."""
    assert r0.tobytes() == r1.tobytes()


def pair(n, a, b, w, h_ids, *, seed=0, K=100.0, T=100, s=32, early_exit=True, ctx_kw=None):
    """A GPU graph and an oracle graph built from the same G(0), H(0)."""
    ctx = D.Context(seed=seed, K=K, T=T, s=s, early_exit=early_exit, **(ctx_kw or {}))
    g = ctx.load_graph(n, a, b, w)
    g.init_sparsifier(a[h_ids], b[h_ids])
    o = OracleGraph(n, a, b, w, seed=seed, K=K, T=T, s=s, early_exit=early_exit)
    o.init_sparsifier(a[h_ids], b[h_ids])
    return ctx, g, o


def step_both(g, o, u, v, w, op, *, check_graphs=True, where=""):
    ups = D.make_updates(u, v, w, op)
    res = g.apply(ups)
    ref = o.apply(u, v, w, op, prune_bounds=g.ctx.del_prune)
    assert_results_equal(res, ref, where)
    if check_graphs:
        assert_edges_equal(g.sparsifier(), o.edges("H"), f"{where} H")
        assert_edges_equal(g.edges(), o.edges("G"), f"{where} G")
    return res, ref
