"""Shared helpers of the GPU parity tests: run the same seeded input through the
CUDA library and through the CPU oracle and compare element by element."""
from __future__ import annotations

import numpy as np

from oracle.oracle import OracleGraph
from paper_2505_02741_b300 import dygrass as D

FIELDS = ("status", "walked", "hit", "accepted", "fallback", "nhits", "best_walker", "nrecovered", "steps")


def assert_results_equal(gpu: np.ndarray, orc: dict, where=""):
    """Exact comparison.  When the oracle ran with prune_bounds (the GPU prunes
    deletion walkers), nhits is compared with its pruned count and steps must
    lie between the exact pruned and unpruned step counts (a pruned walker stops
    somewhere in between, depending on when the better hit became visible)."""
    pruned = "nhits_min" in orc
    for f in FIELDS:
        g = np.asarray(gpu[f]).astype(np.int64)
        if pruned and f == "steps":
            lo = np.asarray(orc["steps_lo"]).astype(np.int64)
            hi = np.asarray(orc["steps"]).astype(np.int64)
            bad = np.nonzero((g < lo) | (g > hi))[0][:10]
            if bad.size:
                raise AssertionError(f"{where} steps outside [pruned, unpruned] at {bad.tolist()}: gpu "
                                     f"{g[bad].tolist()} lo {lo[bad].tolist()} hi {hi[bad].tolist()}")
            continue
        o = np.asarray(orc["nhits_min" if pruned and f == "nhits" else f]).astype(np.int64)
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


def assert_same_outputs(r0: np.ndarray, r1: np.ndarray, steps=True):
    """Two GPU result arrays: every byte, or every field but steps (pruned
    deletion walkers make steps depend on scheduling)."""
    if steps:
        assert r0.tobytes() == r1.tobytes()
        return
    for f in r0.dtype.names:
        if f == "steps":
            continue
        a, b = np.asarray(r0[f]), np.asarray(r1[f])
        if a.dtype.kind == "f":
            a, b = a.view(np.uint64), b.view(np.uint64)
        assert np.array_equal(a, b), f


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
