"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test names the part of the paper (or the published definition) that fixes
the expected value.  None of these needs a GPU.
"""
from __future__ import annotations

import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import checks
from oracle.oracle import (STOP_AT_T, STOP_CUT, STOP_HIT, STOP_LEAF, STOP_OVER_K, OracleGraph,
                           philox4x32_10)
from paper_2505_02741_b300 import workloads as W
from tests.helpers import ReferenceStream, path_graph, random_connected, random_tree, ring

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ---------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            vals = [int(x, 16) for x in line.split()]
            rows.append((vals[0:4], vals[4:6], vals[6:10]))
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    ctr, key, want = row
    assert list(philox4x32_10(ctr, key)) == want


def test_philox_matches_independent_engine():
    """Cross-check against PyTorch's own Philox4x32-10 engine (a separate
    implementation, compiled here on the CPU from its header)."""
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not (shutil.which("g++") and os.path.exists(hdr)):
        pytest.skip("g++ or the PyTorch Philox header is not available")
    rng = np.random.default_rng(7)
    cases = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64)
    src = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long c0, c1, c2, c3, k0, k1;
  while (scanf("%llu %llu %llu %llu %llu %llu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    at::Philox4_32 e(k0 | (k1 << 32), c2 | (c3 << 32), c0 | (c1 << 32));
    unsigned a = e(), b = e(), c = e(), d = e();
    printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        cpp = os.path.join(td, "p.cpp")
        exe = os.path.join(td, "p")
        open(cpp, "w").write(src)
        try:
            subprocess.check_call(["g++", "-std=c++17", "-O1", "-I" + inc, cpp, "-o", exe],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            pytest.skip("PyTorch Philox header does not compile standalone here")
        inp = "\n".join(" ".join(str(int(x)) for x in c) for c in cases) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    got_ref = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()])
    for c, ref in zip(cases, got_ref):
        mine = philox4x32_10([int(c[0]), int(c[1]), int(c[2]), int(c[3])], [int(c[4]), int(c[5])])
        assert list(mine) == list(ref)


def test_philox_uniformity():
    """Word 0 over consecutive step counters is uniform (chi-square, 64 bins)."""
    vals = np.array([philox4x32_10([t, 3, 11, 0], [5, 0])[0] for t in range(20000)], np.uint64)
    counts = np.bincount((vals >> np.uint64(26)).astype(np.int64), minlength=64)
    expected = len(vals) / 64.0
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 120.0  # 63 dof: p ~ 1e-5


# ---------------------------------------------------------------------------
# the non-backtracking sampler (Section III-B)
# ---------------------------------------------------------------------------
def _sampler_graph():
    rng = np.random.default_rng(3)
    a, b, w = random_connected(8, 6, rng)
    # vertex 8 is isolated: a target no walk can reach, so walks run to T or a leaf
    return 9, a, b, w


def test_sampler_matches_enumeration():
    """Empirical path frequencies == exact NBRW probabilities (prod 1/n_eff)."""
    n, a, b, w = _sampler_graph()
    T = 4
    g = OracleGraph(n, a, b, w, T=T, s=1, K=1e300)
    adj = checks.adjacency_lists(n, a, b, w)
    for p in (0, 3):
        exact = checks.enumerate_nb_walks(adj, p, 8, T)
        N = 20000
        freq = {}
        for i in range(N):
            reason, steps, R, path = g.walk(p, 8, 1.0, True, upd_id=i, walker=i % 7, on_h=False)
            key = tuple(int(x) for x in path)
            assert key in exact, f"sampled walk {key} is not a non-backtracking walk"
            assert reason in (STOP_AT_T, STOP_LEAF)
            freq[key] = freq.get(key, 0) + 1
        for key, prob in exact.items():
            sigma = math.sqrt(N * prob * (1 - prob)) + 1e-9
            assert abs(freq.get(key, 0) - N * prob) <= 5 * sigma + 1, (key, prob)


def test_walker_never_backtracks_and_reads_fresh_randoms():
    n, a, b, w = _sampler_graph()
    g = OracleGraph(n, a, b, w, T=50, s=1, K=1e300)
    adj = checks.adjacency_lists(n, a, b, w)
    nbrs = [set(y for y, _ in L) for L in adj]
    for i in range(300):
        _, steps, _, path = g.walk(1, 8, 1.0, True, upd_id=i, walker=0, on_h=False)
        for t in range(steps):
            assert int(path[t + 1]) in nbrs[int(path[t])]
            if t > 0:
                assert path[t + 1] != path[t - 1]


def test_tree_walk_is_unique_path():
    """On a tree the NBRW reaching q follows the unique path, so its resistance is
    R_eff exactly (Section III-B); summed in path order it is bit-identical."""
    rng = np.random.default_rng(11)
    n = 14
    a, b, w = random_tree(n, rng)
    adj = checks.adjacency_lists(n, a, b, w)
    wmap = {(int(x), int(y)): ww for x, y, ww in zip(a, b, w)}
    g = OracleGraph(n, a, b, w, T=100, s=32)
    hits = 0
    for p, q in [(0, 5), (3, 9), (12, 1), (7, 13)]:
        tp = checks.tree_path(adj, p, q)
        R_path = 0.0
        for x, y in zip(tp[:-1], tp[1:]):
            R_path = R_path + 1.0 / wmap[(min(x, y), max(x, y))]
        R_eff = checks.effective_resistance(n, a, b, w, p, q)
        assert R_path == pytest.approx(R_eff, rel=1e-12)
        for k in range(64):
            reason, steps, R, path = g.walk(p, q, 1.0, True, upd_id=100 + k, walker=k, on_h=False)
            if reason == STOP_HIT:
                hits += 1
                assert list(path) == tp
                assert R == R_path  # 0 ULP
    assert hits > 0


def test_hits_upper_bound_effective_resistance():
    """Any walk reaching q has resistance >= R_eff(p, q) (Section III-B)."""
    rng = np.random.default_rng(5)
    n = 12
    a, b, w = random_connected(n, 14, rng, 0.2, 5.0)
    g = OracleGraph(n, a, b, w, T=60, s=32)
    pairs = [(int(x), int(y)) for x, y in rng.integers(0, n, size=(25, 2)) if x != y]
    reff = checks.effective_resistances(n, a, b, w, pairs)
    nh = 0
    for (p, q), re in zip(pairs, reff):
        for k in range(32):
            reason, _, R, _ = g.walk(p, q, 1.0, True, upd_id=7, walker=k, on_h=False)
            if reason == STOP_HIT:
                nh += 1
                assert R >= re * (1 - 1e-12)
    assert nh > 0


# ---------------------------------------------------------------------------
# insertion rule (Section III-B, Algorithm 1 lines 5-9)
# ---------------------------------------------------------------------------
def _line_with_target(L):
    """H = path 0-1-...-L; G = H; insertion (0, L)."""
    a, b, w = path_graph(L + 1)
    return L + 1, a, b, w


@pytest.mark.parametrize("K,T,accepted", [
    (4.0, 100, 0),       # distortion exactly K counts as reachable (case study: K=4 <-> 4 steps)
    (3.999, 100, 1),     # just below: q lies beyond the threshold -> kept
    (100.0, 3, 1),       # step limit before q -> conservatively kept
    (100.0, 4, 0),       # reached on step T counts
])
def test_insertion_forced_path(K, T, accepted):
    n, a, b, w = _line_with_target(4)
    g = OracleGraph(n, a, b, w, K=K, T=T, s=8)
    g.init_sparsifier(a, b)
    r = g.apply([0], [4], [1.0], [0], walkers=True)
    assert r["status"][0] == 0 and r["walked"][0] == 1
    assert r["accepted"][0] == accepted
    assert r["hit"][0] == 1 - accepted
    ha, hb, _ = g.edges("H")
    assert ((0, 4) in set(zip(ha.tolist(), hb.tolist()))) == bool(accepted)
    if not accepted:
        assert r["r_est"][0] == 4.0 and r["nhits"][0] == 8 and r["best_walker"][0] == 0
        assert r["steps"][0] == 8 * 4
    else:
        assert math.isinf(r["r_est"][0]) and r["best_walker"][0] == -1


def test_insertion_distortion_uses_new_edge_weight():
    """w_pq * R > K stops the walker: a heavy new edge is kept, a light one pruned."""
    n, a, b, w = _line_with_target(4)  # R(0->4) = 4
    g = OracleGraph(n, a, b, w, K=10.0, T=100, s=4)
    g.init_sparsifier(a, b)
    r = g.apply([0, 0], [4, 3], [3.0, 2.0], [0, 0])  # 3*4 = 12 > 10 -> keep; 2*3 = 6 <= 10 -> prune
    assert r["accepted"].tolist() == [1, 0]
    assert r["r_est"][1] == 3.0


def test_insertion_unreachable_component_is_kept():
    a = np.array([0, 2], np.int32)
    b = np.array([1, 3], np.int32)
    g = OracleGraph(4, a, b, np.ones(2), s=4)
    g.init_sparsifier(a, b)
    r = g.apply([0], [3], [1.0], [0], walkers=True)
    assert r["accepted"][0] == 1
    assert (r["walkers"][0]["reason"] == STOP_LEAF).all()  # 0 -> 1 is a leaf


def test_isolated_start_is_zero_steps():
    a = np.array([1], np.int32)
    b = np.array([2], np.int32)
    g = OracleGraph(3, a, b, np.ones(1), s=4)
    g.init_sparsifier(a, b)
    r = g.apply([0], [2], [1.0], [0], walkers=True)
    assert r["accepted"][0] == 1 and r["steps"][0] == 0
    assert (r["walkers"][0]["steps"] == 0).all()


def test_early_exit_reading_keeps_decisions():
    """Reading R8 changes only the truncation, never the accept decision; it
    cannot lower R~ nor raise the step count."""
    wl, st = W.make_grid(24, 24)
    batch = st.next_batch(150, 0)
    outs = []
    for ee in (True, False):
        g = OracleGraph(wl.n, wl.a, wl.b, wl.w, early_exit=ee)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        outs.append(g.apply(batch.u, batch.v, batch.w, batch.op, walkers=True))
    on, off = outs
    assert (on["accepted"] == off["accepted"]).all()
    assert (on["steps"] <= off["steps"]).all()
    assert (on["r_est"] >= off["r_est"]).all()
    cut = on["walkers"]["reason"] == STOP_CUT
    assert cut.any()
    # every cut walker stopped at k*, the step of the first hit of its update
    for i in np.nonzero(cut.any(axis=1))[0]:
        kstar = on["walkers"][i]["steps"][on["walkers"][i]["reason"] == STOP_HIT].min()
        assert (on["walkers"][i]["steps"][cut[i]] == kstar).all()


# ---------------------------------------------------------------------------
# deletion rule (Section III-C, Algorithm 1 lines 10-17)
# ---------------------------------------------------------------------------
def test_deletion_outside_sparsifier_is_noop():
    n = 6
    a, b, w = ring(n)
    keep = ~((a == 2) & (b == 3))
    g = OracleGraph(n, a, b, w)
    g.init_sparsifier(a[keep], b[keep])
    r = g.apply([2], [3], [0.0], [1])
    assert r["status"][0] == 0 and r["walked"][0] == 0
    ha, hb, _ = g.edges("H")
    assert len(ha) == n - 1


@pytest.mark.parametrize("n", [6, 9])
def test_deletion_recovers_other_arc(n):
    """Ring G, H = ring minus (2,3).  Deleting (0,1) from H forces every walk
    from 0 around the arc 0, n-1, ..., 2, 1; of its edges only (2,3) is outside
    H', so exactly that edge is recovered (case study: only path edges not
    already in H are recovered)."""
    a, b, w = ring(n)
    keep = ~((a == 2) & (b == 3))
    g = OracleGraph(n, a, b, w, T=n - 1, s=8)
    g.init_sparsifier(a[keep], b[keep])
    r = g.apply([0], [1], [0.0], [1], paths=True)
    assert r["walked"][0] == 1 and r["hit"][0] == 1 and r["fallback"][0] == 0
    assert r["nrecovered"][0] == 1
    assert r["r_est"][0] == float(n - 1)
    ha, hb, _ = g.edges("H")
    hs = set(zip(ha.tolist(), hb.tolist()))
    assert (2, 3) in hs and (0, 1) not in hs and len(hs) == n - 1
    assert r["paths"][0, 0].tolist() == [0] + list(range(n - 1, 0, -1))


def test_deletion_fallback_rule():
    """No walker reaches q within T: each endpoint gets its minimum-resistance
    G_b edge that is not in H' (ties: smaller neighbour id)."""
    # star-ish graph: 0-1 in H (deleted); 0 has G edges to 2 (w 4), 3 (w 4), 4 (w 1);
    # 1 has G edges to 5 (w 2) in H and 6 (w 3) not in H.  H = {01, 15, 04}
    a = np.array([0, 0, 0, 0, 1, 1], np.int32)
    b = np.array([1, 2, 3, 4, 5, 6], np.int32)
    w = np.array([1.0, 4.0, 4.0, 1.0, 2.0, 3.0])
    g = OracleGraph(7, a, b, w, T=3, s=4)
    g.init_sparsifier(np.array([0, 1, 0], np.int32), np.array([1, 5, 4], np.int32))
    r = g.apply([0], [1], [0.0], [1])
    assert r["walked"][0] == 1 and r["hit"][0] == 0 and r["fallback"][0] == 1
    assert r["nrecovered"][0] == 2
    ha, hb, hw = g.edges("H")
    hs = set(zip(ha.tolist(), hb.tolist()))
    # 0: candidates not in H' are (0,2) r=.25 and (0,3) r=.25 -> tie -> smaller id 2
    # 1: candidate not in H' is (1,6)
    assert hs == {(0, 2), (0, 4), (1, 5), (1, 6)}


def test_fallback_rule_long_lists_brute_force():
    """With a step limit of 1 no walker can reach the far endpoint of a deleted
    edge (the edge is gone from G_b and there are no parallel edges), so every
    deletion of an H edge falls back.  H_b must then be H' plus, for each
    endpoint of each deletion, its minimum-resistance G_b edge outside H'
    (ties: smaller neighbour id).  Computed here by brute force on two hubs of
    3000 and 1500 neighbours whose minimum resistance is tied at several
    positions of the list, and on the ring vertices at the other end."""
    rng = np.random.default_rng(31)
    n = 5000
    edges = {}
    for i in range(2, n):  # ring over 2..n-1, all in H
        j = 2 + (i - 2 + 1) % (n - 2)
        edges[(min(i, j), max(i, j))] = True
    for h, d in ((0, 3000), (1, 1500)):
        for y in rng.choice(np.arange(2, n), d, replace=False):
            edges[(h, int(y))] = bool(rng.random() < 0.3)
    edges[(0, 1)] = True
    keys = sorted(edges)
    a = np.array([k[0] for k in keys], np.int32)
    b = np.array([k[1] for k in keys], np.int32)
    in_h = np.array([edges[k] for k in keys])
    w = rng.uniform(0.1, 10.0, a.size)
    for h, ties in ((0, 5), (1, 3)):  # tied minimum resistance outside H, spread over the list
        idx = np.nonzero((a == h) & (b >= 2) & ~in_h)[0]
        w[rng.choice(idx, ties, replace=False)] = 20.0
    g = OracleGraph(n, a, b, w, T=1, s=4)
    g.init_sparsifier(a[in_h], b[in_h])
    dels = rng.choice(np.nonzero(in_h & (a <= 1) & (b >= 2))[0], 150, replace=False)
    du, dv = a[dels].copy(), b[dels].copy()
    flip = rng.random(dels.size) < 0.5
    du[flip], dv[flip] = dv[flip], du[flip]
    du, dv = np.append(du, 0), np.append(dv, 1)
    r = g.apply(du, dv, np.zeros(du.size), np.ones(du.size, np.int32))
    assert (r["walked"] == 1).all() and (r["hit"] == 0).all() and (r["fallback"] == 1).all()
    # brute force
    deleted = {(min(x, y), max(x, y)) for x, y in zip(du.tolist(), dv.tolist())}
    wt = {k: float(x) for k, x in zip(keys, w)}
    gb = {k for k in keys if k not in deleted}
    hp = {k for k in keys if edges[k] and k not in deleted}
    nbrs = {}
    for x, y in gb:
        nbrs.setdefault(x, []).append(y)
        nbrs.setdefault(y, []).append(x)
    expect = set(hp)
    for i, (u, v) in enumerate(zip(du.tolist(), dv.tolist())):
        picked = 0
        for x in (u, v):
            cand = [(1.0 / wt[(min(x, y), max(x, y))], y) for y in nbrs.get(x, [])
                    if (min(x, y), max(x, y)) not in hp]
            if cand:
                _, y = min(cand)
                expect.add((min(x, y), max(x, y)))
                picked += 1
        assert r["nrecovered"][i] == picked
    ha, hb, hw = g.edges("H")
    got = set(zip(ha.tolist(), hb.tolist()))
    assert got == expect
    assert all(float(x) == wt[(int(p), int(q))] for p, q, x in zip(ha, hb, hw))


# ---------------------------------------------------------------------------
# Algorithm 1 and the batch snapshot, restated independently in Python
# ---------------------------------------------------------------------------
def _mixed_stream(rng, n, a, b, count, invalid=True):
    """Random mix of inserts/deletes on an n-vertex graph incl. invalid ones."""
    cur = set(zip(a.tolist(), b.tolist()))
    ups = []
    for _ in range(count):
        r = rng.random()
        if r < 0.45:
            x, y = (int(t) for t in rng.integers(0, n, 2))
            ups.append((x, y, float(rng.uniform(0.5, 5.0)), 0))
        elif r < 0.9 and cur:
            x, y = sorted(cur)[int(rng.integers(0, len(cur)))]
            if rng.random() < 0.5:
                x, y = y, x
            ups.append((x, y, 0.0, 1))
        elif invalid:
            kind = int(rng.integers(0, 4))
            if kind == 0:
                ups.append((1, 1, 1.0, 0))
            elif kind == 1:
                ups.append((n + 3, 0, 1.0, 1))
            elif kind == 2:
                ups.append((0, 2, -1.0, 0))
            else:
                ups.append((0, 2, 1.0, 7))
        else:
            continue
        x, y, _, op = ups[-1]
        if 0 <= x < n and 0 <= y < n and x != y:
            k = (min(x, y), max(x, y))
            if op == 0:
                cur.add(k)
            elif op == 1:
                cur.discard(k)
    return ups


def _compare(ref_res, orc_res):
    for i, r in enumerate(ref_res):
        for k, v in r.items():
            if k == "walkers_lo":  # compared walker by walker by the caller
                continue
            got = orc_res[k][i]
            if isinstance(v, float) and math.isinf(v):
                assert math.isinf(got), (i, k)
            else:
                assert got == v, (i, k, got, v)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sequential_algorithm1(seed):
    """Batches of one update == Algorithm 1 applied update by update."""
    rng = np.random.default_rng(seed)
    n = 16
    a, b, w = random_connected(n, 12, rng)
    h = W.init_sparsifier(n, a, b, w, rng)
    ups = _mixed_stream(rng, n, a, b, 80)
    g = OracleGraph(n, a, b, w, T=12, s=6, K=8.0)
    g.init_sparsifier(a[h], b[h])
    ref = ReferenceStream(n, a, b, w, list(zip(a[h].tolist(), b[h].tolist())), T=12, s=6, K=8.0)
    for up in ups:
        out = g.apply([up[0]], [up[1]], [up[2]], [up[3]])
        _compare(ref.apply([up]), out)
        for which in ("H", "G"):
            ga, gb, gw = g.edges(which)
            ra, rb, rw = ref.edges(which)
            assert ga.tolist() == ra.tolist() and gb.tolist() == rb.tolist()
            assert gw.tolist() == rw.tolist()


@pytest.mark.parametrize("seed", [4, 5])
def test_batch_snapshot(seed):
    """Batches with repeated edges (insert/delete/insert of one pair) follow the
    snapshot reading: validate in order, walk on one snapshot, set-union commit."""
    rng = np.random.default_rng(seed)
    n = 20
    a, b, w = random_connected(n, 16, rng)
    h = W.init_sparsifier(n, a, b, w, rng)
    g = OracleGraph(n, a, b, w, T=10, s=5, K=6.0)
    g.init_sparsifier(a[h], b[h])
    ref = ReferenceStream(n, a, b, w, list(zip(a[h].tolist(), b[h].tolist())), T=10, s=5, K=6.0)
    ups = _mixed_stream(rng, n, a, b, 120)
    # force same-pair sequences inside one batch
    x, y = int(a[h][0]), int(b[h][0])
    ups[10:10] = [(x, y, 0.0, 1), (y, x, 2.5, 0), (x, y, 0.0, 1), (x, y, 3.5, 0)]
    for lo in range(0, len(ups), 31):
        chunk = ups[lo:lo + 31]
        cols = list(zip(*chunk))
        out = g.apply(list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]))
        _compare(ref.apply(chunk), out)
        for which in ("H", "G"):
            ga, gb, gw = g.edges(which)
            ra, rb, rw = ref.edges(which)
            assert ga.tolist() == ra.tolist() and gb.tolist() == rb.tolist()
            assert gw.tolist() == rw.tolist()
    assert g.next_id == len(ups)


@pytest.mark.parametrize("seed", [6, 7, 8])
def test_deletion_pruning_bounds(seed):
    """nhits_min / steps_lo of walked deletions (walkers stopping once their
    resistance passes R~) against a restatement that re-sums each walker's
    resistance along its path; unit weights make equal resistances common, so
    ties at R~ are exercised too."""
    rng = np.random.default_rng(seed)
    n = 24
    a, b, w = random_connected(n, 30, rng, unit=(seed == 8))
    h = W.init_sparsifier(n, a, b, w, rng, frac=0.3)
    g = OracleGraph(n, a, b, w, T=16, s=8, K=10.0)
    g.init_sparsifier(a[h], b[h])
    ref = ReferenceStream(n, a, b, w, list(zip(a[h].tolist(), b[h].tolist())), T=16, s=8, K=10.0,
                          prune_bounds=True)
    ups = _mixed_stream(rng, n, a, b, 150, invalid=False)
    pruned = 0
    for lo in range(0, len(ups), 25):
        chunk = ups[lo:lo + 25]
        cols = list(zip(*chunk))
        out = g.apply(list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]), prune_bounds=True,
                      walkers=True)
        rr = ref.apply(chunk)
        _compare(rr, out)
        # every walker's record under the cut: stop reason and step count
        for i, r in enumerate(rr):
            if not r["walked"]:
                continue
            assert [tuple(x) for x in r["walkers_lo"]] == \
                [(int(x["reason"]), int(x["steps"])) for x in out["walkers_lo"][i]], (lo, i)
        assert (out["walkers_lo"]["steps"].sum(axis=1) == out["steps_lo"]).all()
        assert (out["steps_lo"] <= out["steps"]).all() and (out["nhits_min"] <= out["nhits"]).all()
        pruned += int((out["steps"] - out["steps_lo"]).sum())
    assert pruned > 0


@pytest.mark.parametrize("threads", [2, 4])
def test_openmp_build_gives_identical_outputs(threads):
    """The OpenMP build of the oracle runs the walks of a batch's updates on
    several host threads; every output (results, walker records, paths, the
    pruned counts, H and G) equals the single-threaded build's, batch after
    batch."""
    wl, st = W.make_grid(24, 24)
    one = OracleGraph(wl.n, wl.a, wl.b, wl.w, T=60)
    many = OracleGraph(wl.n, wl.a, wl.b, wl.w, T=60, threads=threads)
    assert many.threads == threads and one.threads == 1
    for g in (one, many):
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for _ in range(3):
        bt = st.next_batch(80, 60)
        r1 = one.apply(bt.u, bt.v, bt.w, bt.op, walkers=True, paths=True, prune_bounds=True)
        r2 = many.apply(bt.u, bt.v, bt.w, bt.op, walkers=True, paths=True, prune_bounds=True)
        assert r1.keys() == r2.keys()
        for k in r1:
            assert np.asarray(r1[k]).tobytes() == np.asarray(r2[k]).tobytes(), k
        for which in ("H", "G"):
            for x, y in zip(one.edges(which), many.edges(which)):
                assert x.tobytes() == y.tobytes()


def test_invariants_after_stream():
    """H stays a subgraph of G with G's weights; on the grid with insertions and
    deletions, H keeps the components of G."""
    wl, st = W.make_grid(24, 24)
    g = OracleGraph(wl.n, wl.a, wl.b, wl.w, T=100)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    for _ in range(3):
        bt = st.next_batch(60, 40)
        out = g.apply(bt.u, bt.v, bt.w, bt.op)
        assert (out["status"] == 0).all()
        ga, gb, gw = g.edges("G")
        ha, hb, hw = g.edges("H")
        gmap = dict(zip(zip(ga.tolist(), gb.tolist()), gw.tolist()))
        for x, y, ww in zip(ha.tolist(), hb.tolist(), hw.tolist()):
            assert gmap[(x, y)] == ww
        assert checks.n_components(wl.n, ha, hb) == checks.n_components(wl.n, ga, gb)


# ---------------------------------------------------------------------------
# spectral facts of Section III-B (Eqs. 6-11) and R_eff closed forms
# ---------------------------------------------------------------------------
def test_effective_resistance_series_parallel():
    # 0 -(2)- 1 -(3)- 2 in series, and a parallel 0 -(6)- 2 branch (w = conductance)
    a = np.array([0, 1, 0], np.int32)
    b = np.array([1, 2, 2], np.int32)
    w = np.array([2.0, 3.0, 6.0])
    series = 1 / 2.0 + 1 / 3.0
    par = 1 / 6.0
    want = series * par / (series + par)
    assert checks.effective_resistance(3, a, b, w, 0, 2) == pytest.approx(want, rel=1e-13)
    assert checks.effective_resistance(3, a[:2], b[:2], w[:2], 0, 2) == pytest.approx(series, rel=1e-13)


def test_condition_number_bounds():
    """lambda_min(L_G, L_H) >= 1 for H a spanning subgraph with G's weights, and
    w_e * R_eff,H(e) <= kappa for every edge of G (Eq. 11)."""
    wl, _ = W.make_grid(12, 12)
    hs = (wl.a[wl.h_ids], wl.b[wl.h_ids], wl.w[wl.h_ids])
    ev = checks.pencil_eigs(wl.n, (wl.a, wl.b, wl.w), hs)
    assert ev[0] >= 1 - 1e-9
    kap = ev[-1] / ev[0]
    pairs = list(zip(wl.a.tolist(), wl.b.tolist()))
    rh = checks.effective_resistances(wl.n, *hs, pairs)
    rg = checks.effective_resistances(wl.n, wl.a, wl.b, wl.w, pairs)
    assert (wl.w * rh <= kap * (1 + 1e-9)).all()
    assert (rh / rg <= ev[-1] * (1 + 1e-9)).all()


def test_spanning_forest_is_kruskal():
    rng = np.random.default_rng(9)
    for trial in range(6):
        n = 30
        a, b, w = random_connected(n, 40, rng, unit=(trial % 2 == 0))
        if trial >= 4:  # disconnected: drop a random third of the edges
            keep = rng.random(a.size) > 0.35
            a, b, w = a[keep], b[keep], w[keep]
        ids = W.spanning_forest(n, a, b, w)
        assert ids.tolist() == checks.kruskal_max_forest(n, a, b, w)
        assert ids.size == n - checks.n_components(n, a, b)


def test_initial_sparsifier_rule():
    wl, _ = W.make_grid(64, 64)
    tree = W.spanning_forest(wl.n, wl.a, wl.b, wl.w)
    off = wl.m - tree.size
    assert wl.h_ids.size == tree.size + math.floor(0.1 * off)
    assert np.isin(tree, wl.h_ids).all()


# ---------------------------------------------------------------------------
# GRASS-like initial sparsifier: stretch of the off-tree edges (reading R20)
# ---------------------------------------------------------------------------
def _forest(n, a, b, w):
    return W.spanning_forest(n, a, b, w)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_tree_stretch_is_path_resistance(seed):
    """w_e * R_T(e): R_T against the tree path's resistance summed edge by
    edge and against R_eff of the tree alone (pseudo-inverse), 1e-12
    relative; tree edges read 0."""
    from oracle.oracle import tree_stretch
    rng = np.random.default_rng(seed)
    n = 40
    a, b, w = random_connected(n, 50, rng, 0.2, 7.0)
    tree = _forest(n, a, b, w)
    st = tree_stretch(n, a, b, w, tree)
    mask = np.zeros(a.size, bool)
    mask[tree] = True
    assert (st[mask] == 0.0).all()
    ta, tb, tw = a[mask], b[mask], w[mask]
    adj = checks.adjacency_lists(n, ta, tb, tw)
    off = np.nonzero(~mask)[0]
    pairs = [(int(a[i]), int(b[i])) for i in off]
    reff = checks.effective_resistances(n, ta, tb, tw, pairs)
    for k, i in enumerate(off):
        path = checks.tree_path(adj, int(a[i]), int(b[i]))
        wmap = {(int(x), int(y)): float(z) for x, y, z in zip(ta, tb, tw)}
        rsum = sum(1.0 / wmap[(min(p, q), max(p, q))] for p, q in zip(path[:-1], path[1:]))
        assert st[i] == pytest.approx(w[i] * rsum, rel=1e-12)
        assert st[i] == pytest.approx(w[i] * reff[k], rel=1e-12)


def test_tree_stretch_unit_weights_is_hop_distance():
    """Unit weights: the stretch of a chord of a path is exactly its hop count."""
    from oracle.oracle import tree_stretch
    n = 30
    pa, pb, _ = path_graph(n)
    chords = [(0, 29), (3, 10), (5, 6 + 7), (12, 27)]
    a = np.concatenate([pa, [c[0] for c in chords]]).astype(np.int32)
    b = np.concatenate([pb, [c[1] for c in chords]]).astype(np.int32)
    ca, cb, _ = W.canonical(a, b)
    w = np.ones(ca.size)
    tree = np.nonzero((cb - ca) == 1)[0]
    st = tree_stretch(n, ca, cb, w, tree)
    for x, y, s in zip(ca, cb, st):
        assert s == (0.0 if y - x == 1 else float(y - x))


def test_tree_stretch_across_trees_cycles_and_selection():
    """An off-tree edge between two trees of the forest has infinite stretch;
    marked edges that close a cycle are rejected; the GRASS-like H(0) is the
    forest plus the n_off largest stretches, ties to the smaller edge id."""
    from oracle.oracle import grass_sparsifier, tree_stretch
    a, b, w = ring(8, w=2.0)
    ids = np.arange(a.size)
    with pytest.raises(ValueError):
        tree_stretch(8, a, b, w, ids)  # the whole ring is a cycle
    # forest of two paths {0..3}, {4..7}: edges 3-4 and 0-7 cross between them
    keep = [i for i in ids if not ((a[i], b[i]) in ((3, 4), (0, 7)))]
    st = tree_stretch(8, a, b, w, keep)
    cross = [i for i in ids if (a[i], b[i]) in ((3, 4), (0, 7))]
    assert np.isinf(st[cross]).all()
    rng = np.random.default_rng(5)
    n = 60
    a, b, w = random_connected(n, 80, rng, unit=True)  # unit weights: many equal stretches
    tree = _forest(n, a, b, w)
    st = tree_stretch(n, a, b, w, tree)
    for n_off in (0, 7, 23):
        h = grass_sparsifier(n, a, b, w, tree, n_off)
        off = sorted((i for i in range(a.size) if i not in set(tree.tolist())), key=lambda i: (-st[i], i))
        assert h.tolist() == sorted(tree.tolist() + off[:n_off])
