"""Small-graph builders and a plain-Python restatement of the update rules.

``ReferenceStream`` states Algorithm 1 (insertion / deletion branches) with the
batch-snapshot reading a second time, in plain Python dictionaries and sets,
independently of the C oracle's batch code.  For the walks themselves it calls
the oracle's single-walker routine on a throw-away graph built from its own
sets; that routine is pinned separately (enumeration, tree closed form).
"""
from __future__ import annotations

import math

import numpy as np

from oracle.oracle import STOP_CUT, STOP_HIT, OracleGraph


def random_connected(n, extra, rng, wlo=1.0, whi=10.0, unit=False):
    """Random spanning tree + ``extra`` distinct extra edges; canonical, sorted."""
    edges = set()
    perm = rng.permutation(n)
    for i in range(1, n):
        a, b = int(perm[i]), int(perm[rng.integers(0, i)])
        edges.add((min(a, b), max(a, b)))
    tries = 0
    while len(edges) < n - 1 + extra and tries < 100 * (extra + 1):
        a, b = (int(x) for x in rng.integers(0, n, 2))
        tries += 1
        if a != b:
            edges.add((min(a, b), max(a, b)))
    e = sorted(edges)
    a = np.array([x for x, _ in e], np.int32)
    b = np.array([y for _, y in e], np.int32)
    w = np.ones(len(e)) if unit else rng.uniform(wlo, whi, len(e))
    return a, b, w


def random_tree(n, rng, wlo=0.5, whi=5.0):
    return random_connected(n, 0, rng, wlo, whi)


def ring(n, w=1.0):
    a = np.array([min(i, (i + 1) % n) for i in range(n)], np.int32)
    b = np.array([max(i, (i + 1) % n) for i in range(n)], np.int32)
    order = np.lexsort((b, a))
    return a[order], b[order], np.full(n, w, dtype=np.float64)


def path_graph(n, w=1.0):
    a = np.arange(n - 1, dtype=np.int32)
    return a, a + 1, np.full(n - 1, w, dtype=np.float64)


# ---------------------------------------------------------------------------
# plain restatement of Algorithm 1 + the batch snapshot
# ---------------------------------------------------------------------------
def _key(a, b):
    return (a, b) if a < b else (b, a)


class ReferenceStream:
    def __init__(self, n, a, b, w, h_pairs, *, seed=0, K=100.0, T=100, s=32, early_exit=True,
                 prune_bounds=False):
        self.prune_bounds = prune_bounds
        self.n = n
        self.G = {(int(x), int(y)): float(ww) for x, y, ww in zip(a, b, w)}
        self.H = set(_key(int(x), int(y)) for x, y in h_pairs)
        self.seed, self.K, self.T, self.s, self.early_exit = seed, K, T, s, early_exit
        self.next_id = 0

    def _walker(self, edges_w, u, v, wpq, deletion, upd_id):
        """Run the s walkers of one update on the graph ``edges_w``."""
        items = sorted(edges_w.items())
        a = np.array([k[0] for k, _ in items], np.int32)
        b = np.array([k[1] for k, _ in items], np.int32)
        w = np.array([x for _, x in items], np.float64)
        g = OracleGraph(self.n, a, b, w, seed=self.seed, K=self.K, T=self.T, s=self.s)
        out = [g.walk(u, v, wpq, deletion, upd_id, k, on_h=False) for k in range(self.s)]
        g.close()
        return out

    def apply(self, ups):
        n = self.n
        res = []
        view = dict(self.G)
        h_start = set(self.H)
        hdel = set()
        for (u, v, w, op) in ups:
            r = dict(status=0, walked=0, hit=0, accepted=0, fallback=0, nhits=0, best_walker=-1,
                     nrecovered=0, steps=0, r_est=math.inf)
            if op not in (0, 1):
                r["status"] = 6
            elif not (0 <= u < n and 0 <= v < n):
                r["status"] = 2
            elif u == v:
                r["status"] = 1
            elif op == 0:
                k = _key(u, v)
                if not (math.isfinite(w) and w > 0):
                    r["status"] = 5
                elif k in view:
                    r["status"] = 3
                else:
                    view[k] = w
                    r["walked"] = 1
            else:
                k = _key(u, v)
                if k not in view:
                    r["status"] = 4
                else:
                    del view[k]
                    if k in h_start:
                        r["walked"] = 1
                        hdel.add(k)
            res.append(r)
        Gb = view
        Hp = h_start - hdel
        Hp_w = {k: Gb[k] for k in Hp}
        commits = set()
        for i, (u, v, w, op) in enumerate(ups):
            r = res[i]
            if not r["walked"]:
                continue
            deletion = op == 1
            walks = self._walker(Gb if deletion else Hp_w, u, v, 0.0 if deletion else w, deletion,
                                 self.next_id + i)
            reasons = [x[0] for x in walks]
            steps = [x[1] for x in walks]
            Rs = [x[2] for x in walks]
            paths = [x[3] for x in walks]
            hits = [k for k in range(self.s) if reasons[k] == STOP_HIT]
            if not deletion and self.early_exit and hits:
                kstar = min(steps[k] for k in hits)
                for k in range(self.s):
                    if steps[k] > kstar:
                        steps[k] = kstar
                        reasons[k] = STOP_CUT
                hits = [k for k in range(self.s) if reasons[k] == STOP_HIT]
            r["nhits"] = len(hits)
            r["hit"] = int(bool(hits))
            r["steps"] = int(sum(steps))
            if hits:
                best = min(hits, key=lambda k: (Rs[k], k))
                r["best_walker"] = best
                r["r_est"] = Rs[best]
            if self.prune_bounds:
                # deletion pruning: a walker whose resistance passes R~ cannot give the
                # minimum; its steps end at the first such step, recomputed here from
                # its path and the G_b weights (r = 1/w, summed in walk order)
                r["nhits_min"], r["steps_lo"] = r["nhits"], r["steps"]
                r["walkers_lo"] = list(zip(reasons, steps))
                if deletion and hits:
                    rstar = r["r_est"]
                    lo = 0
                    for k in range(self.s):
                        if k in hits and Rs[k] == rstar:
                            lo += steps[k]
                            continue
                        R, cut = 0.0, steps[k]
                        for t in range(1, steps[k] + 1):
                            R = R + 1.0 / Gb[_key(int(paths[k][t - 1]), int(paths[k][t]))]
                            if R > rstar:
                                cut = t
                                r["walkers_lo"][k] = (STOP_CUT, t)
                                break
                        lo += cut
                    r["nhits_min"] = sum(1 for k in hits if Rs[k] == rstar)
                    r["steps_lo"] = lo
            if not deletion:
                r["accepted"] = int(not hits)
                if r["accepted"] and _key(u, v) in Gb:
                    commits.add(_key(u, v))
                continue
            emitted = set()
            if hits:
                p = paths[r["best_walker"]]
                for t in range(len(p) - 1):
                    k = _key(int(p[t]), int(p[t + 1]))
                    if k not in Hp:
                        emitted.add(k)
            else:
                r["fallback"] = 1
                for x in (u, v):
                    cand = []
                    for k in Gb:
                        if x not in k or k in Hp:
                            continue
                        y = k[1] if k[0] == x else k[0]
                        cand.append((1.0 / Gb[k], y, k))
                    if cand:
                        cand.sort(key=lambda t: (t[0], t[1]))
                        emitted.add(cand[0][2])
            r["nrecovered"] = len(emitted)
            commits |= emitted
        self.G = Gb
        self.H = Hp | commits
        self.next_id += len(ups)
        return res

    def edges(self, which="H"):
        if which == "H":
            items = sorted((k, self.G[k]) for k in self.H)
        else:
            items = sorted(self.G.items())
        a = np.array([k[0] for k, _ in items], np.int32)
        b = np.array([k[1] for k, _ in items], np.int32)
        w = np.array([x for _, x in items], np.float64)
        return a, b, w
