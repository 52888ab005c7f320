"""Seeded synthetic workloads: graphs, initial sparsifiers and update streams.

This module only builds INPUTS.  It holds none of dyGRASS's arithmetic (no
walks, no resistances, no accept/recover rules), so both the CUDA path and the
CPU oracle may consume what it produces.

Every random draw comes from ``numpy.random.Generator(PCG64(SeedSequence(seed)))``
with one spawned child stream per purpose (structure, weights, initial-H sample,
updates, arrivals), so a workload is a pure function of its seed.

Graphs are returned in canonical form: undirected simple edges ``(u, v)`` with
``u < v``, sorted lexicographically; the canonical edge id is the row index.

The paper's benchmark matrices (SuiteSparse circuit, FEA and Delaunay meshes,
Section IV) are not available; the generators below stand in for them:

* ``grid2d``      – 2-D 4-neighbour grid (small parity workload),
* ``mesh3d``      – 3-D power-grid-like mesh with heavier z "via" edges,
* ``fea_tri``     – jittered, randomly triangulated 2-D grid (FEA / Delaunay-like),
* ``rmat``        – symmetrised R-MAT power-law graph (social-network-like).

The initial sparsifier H(0) replaces GRASS (Section III-A, which precomputes it)
by a max-weight spanning forest (Kruskal order: weight descending, ties by edge
id) plus a seeded 10 % sample of the off-tree edges.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import minimum_spanning_tree

OP_INSERT = 0
OP_DELETE = 1

_STREAMS = ("structure", "weights", "init_h", "updates", "arrivals")


def rngs(seed: int) -> dict:
    """One independent PCG64 generator per purpose, spawned from ``seed``."""
    children = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    return {k: np.random.Generator(np.random.PCG64(c)) for k, c in zip(_STREAMS, children)}


# --------------------------------------------------------------------------
# canonical edge lists
# --------------------------------------------------------------------------
def canonical(u, v, w=None):
    """Orient every edge as (min, max) and sort lexicographically."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    span = np.int64(int(b.max()) + 1) if b.size else np.int64(1)
    order = np.argsort(a * span + b, kind="stable")  # (a, b) lexicographic, ties in input order
    a, b = a[order], b[order]
    out_w = None if w is None else np.asarray(w, dtype=np.float64)[order]
    return a.astype(np.int32), b.astype(np.int32), out_w


def edge_keys(n: int, a, b) -> np.ndarray:
    """int64 key a*n+b of canonical pairs (a < b): sorting keys == lexicographic order."""
    return np.asarray(a, dtype=np.int64) * np.int64(n) + np.asarray(b, dtype=np.int64)


def csr_of(n: int, a, b):
    """Symmetric CSR (indptr, indices) of an undirected edge list, neighbours sorted."""
    src = np.concatenate([a, b]).astype(np.int64)
    dst = np.concatenate([b, a]).astype(np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, src + 1, 1)
    np.cumsum(indptr, out=indptr)
    return indptr, dst


# --------------------------------------------------------------------------
# graph families
# --------------------------------------------------------------------------
def grid2d(nx: int, ny: int):
    """4-neighbour grid; vertex id = y*nx + x."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    hu, hv = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    vu, vv = idx[:-1, :].ravel(), idx[1:, :].ravel()
    a, b, _ = canonical(np.concatenate([hu, vu]), np.concatenate([hv, vv]))
    return nx * ny, a, b


def mesh3d(nx: int, ny: int, nz: int):
    """6-neighbour 3-D mesh; returns (n, a, b, is_z) with is_z marking z-direction edges."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    parts_u = [idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()]
    parts_v = [idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()]
    zflag = np.concatenate([np.zeros(parts_u[0].size + parts_u[1].size, dtype=bool),
                            np.ones(parts_u[2].size, dtype=bool)])
    u = np.concatenate(parts_u)
    v = np.concatenate(parts_v)
    order = np.lexsort((v, u))  # already u < v for every part
    return nx * ny * nz, u[order].astype(np.int32), v[order].astype(np.int32), zflag[order]


def fea_tri(nx: int, ny: int, rng: np.random.Generator, jitter: float = 0.3):
    """Jittered grid, every cell split by a random diagonal. Returns (n, a, b, pos)."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    gx, gy = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    pos = np.stack([gx.ravel(), gy.ravel()], axis=1)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    hu, hv = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    vu, vv = idx[:-1, :].ravel(), idx[1:, :].ravel()
    c00 = idx[:-1, :-1].ravel()
    c10 = idx[:-1, 1:].ravel()
    c01 = idx[1:, :-1].ravel()
    c11 = idx[1:, 1:].ravel()
    flip = rng.random(c00.size) < 0.5
    du = np.where(flip, c10, c00)
    dv = np.where(flip, c01, c11)
    a, b, _ = canonical(np.concatenate([hu, vu, du]), np.concatenate([hv, vv, dv]))
    return nx * ny, a, b, pos


def rmat(scale: int, n_edges: int, rng: np.random.Generator,
         abcd=(0.57, 0.19, 0.19, 0.05), round_size: int | None = None):
    """Symmetrised R-MAT: self-loops and duplicates removed, vertex ids permuted.

    Every level of a sample picks a quadrant from one 32-bit draw x: a when
    x < 2^32 a, b below 2^32 (a + b), c below 2^32 (a + b + c), else d.
    Samples are drawn in rounds of ``round_size`` (default min(2^24, 2 n_edges))
    until ``n_edges`` distinct undirected edges exist; the ``n_edges`` distinct
    edges drawn first are kept.
    """
    n = 1 << scale
    if scale > 31:
        raise ValueError("scale <= 31")
    ta, tab, tabc = (np.uint32(min(int(round(x * 2.0 ** 32)), 2 ** 32 - 1)) for x in np.cumsum(abcd)[:3])
    m = round_size if round_size else min(1 << 24, max(1 << 16, 2 * n_edges))
    u = np.empty(m, np.uint32)
    v = np.empty(m, np.uint32)
    t1 = np.empty(m, bool)
    t2 = np.empty(m, bool)
    uniq = np.empty(0, np.int64)   # distinct canonical keys so far (sorted)
    first = np.empty(0, np.int64)  # draw position of each key's first sample
    base = 0
    while uniq.size < n_edges:
        u[:] = 0
        v[:] = 0
        for _ in range(scale):
            x = rng.integers(0, 2 ** 32 - 1, size=m, dtype=np.uint32, endpoint=True)
            np.left_shift(u, 1, out=u)
            np.greater_equal(x, tab, out=t1)          # quadrant c or d: row bit
            np.bitwise_or(u, t1, out=u)
            np.left_shift(v, 1, out=v)
            np.greater_equal(x, ta, out=t1)
            np.less(x, tab, out=t2)
            np.logical_and(t1, t2, out=t1)            # quadrant b ...
            np.greater_equal(x, tabc, out=t2)         # ... or d: column bit
            np.logical_or(t1, t2, out=t1)
            np.bitwise_or(v, t1, out=v)
        keep = u != v
        uu = u[keep].astype(np.int64)
        vv = v[keep].astype(np.int64)
        k = np.minimum(uu, vv) * n + np.maximum(uu, vv)
        ku, kf = np.unique(k, return_index=True)
        kf += base
        base += k.size
        if uniq.size:
            pos = np.searchsorted(uniq, ku)
            new = uniq[np.minimum(pos, uniq.size - 1)] != ku
            ku, kf, pos = ku[new], kf[new], pos[new]
            uniq = np.insert(uniq, pos, ku)
            first = np.insert(first, pos, kf)
        else:
            uniq, first = ku, kf
    if uniq.size > n_edges:  # the n_edges keys drawn first (draw positions are distinct)
        uniq = uniq[np.sort(np.argpartition(first, n_edges - 1)[:n_edges])]
    perm = rng.permutation(n).astype(np.int64)
    a, b = perm[uniq // n], perm[uniq % n]
    keys = np.sort(np.minimum(a, b) * n + np.maximum(a, b))
    return n, (keys // n).astype(np.int32), (keys % n).astype(np.int32)


# --------------------------------------------------------------------------
# initial sparsifier
# --------------------------------------------------------------------------
def spanning_forest(n: int, a, b, w) -> np.ndarray:
    """Edge ids of the max-weight spanning forest, Kruskal order (w desc, id asc).

    Each edge gets a distinct rank weight (1 + its position in Kruskal order), so
    the minimum spanning forest under those ranks is unique and equals the forest
    Kruskal's algorithm builds when it scans edges in that order.
    """
    m = len(a)
    order = np.lexsort((np.arange(m), -np.asarray(w)))
    rank = np.empty(m, dtype=np.float64)
    rank[order] = np.arange(1, m + 1, dtype=np.float64)
    mat = sp.csr_matrix((rank, (np.asarray(a, np.int64), np.asarray(b, np.int64))), shape=(n, n))
    t = minimum_spanning_tree(mat).tocoo()
    ids = order[(t.data.astype(np.int64) - 1)]
    return np.sort(ids)


def init_sparsifier(n: int, a, b, w, rng: np.random.Generator, frac: float = 0.1) -> np.ndarray:
    """Spanning forest + exactly floor(frac * #off-tree) off-tree edges (no replacement)."""
    tree = spanning_forest(n, a, b, w)
    mask = np.ones(len(a), dtype=bool)
    mask[tree] = False
    off = np.nonzero(mask)[0]
    k = int(np.floor(frac * off.size))
    pick = np.sort(rng.choice(off, size=k, replace=False)) if k > 0 else np.empty(0, np.int64)
    return np.sort(np.concatenate([tree, pick]))


# --------------------------------------------------------------------------
# update streams
# --------------------------------------------------------------------------
@dataclass
class Batch:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    op: np.ndarray

    def __len__(self):
        return int(self.u.size)


@dataclass
class Workload:
    name: str
    n: int
    a: np.ndarray          # canonical edges of G(0)
    b: np.ndarray
    w: np.ndarray
    h_ids: np.ndarray      # edge ids of H(0)
    K: float = 100.0
    T: int = 100
    s: int = 32
    seed: int = 0
    pos: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.a.size)


class UpdateStream:
    """Generates successive batches against the evolving edge set of G.

    ``ins_rule`` decides how insertion endpoints are drawn:
      * ("hops", hmin, hmax): u uniform, v = end of a simple random walk of
        h ~ U{hmin..hmax} steps in G(0); rejected when v == u, when (u, v) is a
        current edge, or when repeated inside the batch;
      * ("uniform",): u != v uniform, rejected when a current edge or repeated.
    ``w_rule`` maps (rng, u, v) -> weights of the inserted edges.
    Deletions are drawn uniformly without replacement from the current edges at
    the start of the batch.  Insertions and deletions are shuffled together.
    """

    def __init__(self, wl: Workload, rng: np.random.Generator, ins_rule, w_rule):
        self.wl = wl
        self.rng = rng
        self.ins_rule = ins_rule
        self.w_rule = w_rule
        self.n = wl.n
        self.cur = edge_keys(wl.n, wl.a, wl.b)  # sorted (canonical order)
        self._csr = None

    def _csr0(self):
        if self._csr is None:
            self._csr = csr_of(self.wl.n, self.wl.a, self.wl.b)
        return self._csr

    def _is_edge(self, keys):
        pos = np.searchsorted(self.cur, keys)
        pos = np.minimum(pos, self.cur.size - 1)
        return (self.cur.size > 0) & (self.cur[pos] == keys)

    def _draw_inserts(self, count: int):
        rng, n = self.rng, self.n
        got_a, got_b = [], []
        seen = np.empty(0, dtype=np.int64)
        need = count
        while need > 0:
            m = max(64, 2 * need)
            if self.ins_rule[0] == "hops":
                hmin, hmax = self.ins_rule[1], self.ins_rule[2]
                indptr, indices = self._csr0()
                c = rng.integers(0, n, size=m)
                start = c.copy()
                hops = rng.integers(hmin, hmax + 1, size=m)
                for step in range(hmax):
                    act = hops > step
                    deg = indptr[c + 1] - indptr[c]
                    r = rng.random(m)
                    ok = act & (deg > 0)
                    pick = indptr[c] + np.minimum((r * np.maximum(deg, 1)).astype(np.int64),
                                                  np.maximum(deg - 1, 0))
                    c = np.where(ok, indices[np.minimum(pick, indices.size - 1)], c)
                u, v = start, c
            else:
                u = rng.integers(0, n, size=m)
                v = rng.integers(0, n, size=m)
            keep = u != v
            u, v = u[keep], v[keep]
            a, b = np.minimum(u, v), np.maximum(u, v)
            k = edge_keys(n, a, b)
            keep = ~self._is_edge(k)
            u, v, k = u[keep], v[keep], k[keep]
            # drop repeats (within this draw and against earlier draws), keep first
            _, first = np.unique(k, return_index=True)
            first = np.sort(first)
            u, v, k = u[first], v[first], k[first]
            keep = ~np.isin(k, seen)
            u, v, k = u[keep], v[keep], k[keep]
            u, v, k = u[:need], v[:need], k[:need]
            got_a.append(u)
            got_b.append(v)
            seen = np.concatenate([seen, k])
            need -= u.size
        return np.concatenate(got_a).astype(np.int32), np.concatenate(got_b).astype(np.int32)

    def next_batch(self, n_ins: int, n_del: int) -> Batch:
        rng, n = self.rng, self.n
        iu, iv = self._draw_inserts(n_ins) if n_ins > 0 else (np.empty(0, np.int32),) * 2
        iw = self.w_rule(rng, iu, iv) if n_ins > 0 else np.empty(0)
        n_del = min(n_del, self.cur.size)
        didx = np.sort(rng.choice(self.cur.size, size=n_del, replace=False)) if n_del > 0 \
            else np.empty(0, np.int64)
        dk = self.cur[didx]
        du, dv = (dk // n).astype(np.int32), (dk % n).astype(np.int32)
        # randomly orient deletions so both endpoints act as the walk start
        flip = rng.random(n_del) < 0.5
        du, dv = np.where(flip, dv, du), np.where(flip, du, dv)
        u = np.concatenate([iu, du]).astype(np.int32)
        v = np.concatenate([iv, dv]).astype(np.int32)
        w = np.concatenate([np.asarray(iw, np.float64), np.zeros(n_del)])
        op = np.concatenate([np.full(n_ins, OP_INSERT, np.int32), np.full(n_del, OP_DELETE, np.int32)])
        perm = rng.permutation(u.size)
        # advance the tracked edge set
        keep = np.ones(self.cur.size, dtype=bool)
        keep[didx] = False
        ik = np.sort(edge_keys(n, np.minimum(iu, iv), np.maximum(iu, iv)))
        kept = self.cur[keep]
        # inserted keys are distinct and absent from the current set: a sorted insert keeps it sorted
        self.cur = np.insert(kept, np.searchsorted(kept, ik), ik)
        return Batch(u[perm], v[perm], w[perm], op[perm])


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def _u1_10(rng, u, v):
    return rng.uniform(1.0, 10.0, size=len(u))


def _logu(rng, u, v):
    return 10.0 ** rng.uniform(-2.0, 2.0, size=len(u))


def make_grid(nx: int = 64, ny: int = 64, seed: int = 0, K: float = 100.0, T: int = 100,
              s: int = 32) -> tuple[Workload, UpdateStream]:
    """Small parity workload: 2-D grid, w ~ U[1,10], insertions <= 4 hops apart."""
    r = rngs(seed)
    n, a, b = grid2d(nx, ny)
    w = r["weights"].uniform(1.0, 10.0, size=a.size)
    h = init_sparsifier(n, a, b, w, r["init_h"])
    wl = Workload(f"grid2d_{nx}x{ny}", n, a, b, w, h, K=K, T=T, s=s, seed=seed)
    return wl, UpdateStream(wl, r["updates"], ("hops", 2, 4), _u1_10)


def make_mesh3d(nx: int = 100, ny: int = 100, nz: int = 100, seed: int = 0, K: float = 100.0,
                T: int = 100, s: int = 32) -> tuple[Workload, UpdateStream]:
    """Power-grid-like 3-D mesh: w = 10^U(-2,2), z (via) edges 5x heavier;
    insertions <= 6 hops apart with the same (non-z) weight law."""
    r = rngs(seed)
    n, a, b, isz = mesh3d(nx, ny, nz)
    w = 10.0 ** r["weights"].uniform(-2.0, 2.0, size=a.size)
    w = np.where(isz, 5.0 * w, w)
    h = init_sparsifier(n, a, b, w, r["init_h"])
    wl = Workload(f"mesh3d_{nx}x{ny}x{nz}", n, a, b, w, h, K=K, T=T, s=s, seed=seed)
    return wl, UpdateStream(wl, r["updates"], ("hops", 2, 6), _logu)


def make_fea(nx: int = 2048, ny: int = 2048, seed: int = 0, K: float = 100.0, T: int = 100,
             s: int = 32) -> tuple[Workload, UpdateStream]:
    """FEA-like triangulated jittered grid: w = 1/edge length; insertions <= 4 hops
    apart with w = 1/length."""
    r = rngs(seed)
    n, a, b, pos = fea_tri(nx, ny, r["structure"])
    w = 1.0 / np.linalg.norm(pos[a] - pos[b], axis=1)
    h = init_sparsifier(n, a, b, w, r["init_h"])
    wl = Workload(f"fea_tri_{nx}x{ny}", n, a, b, w, h, K=K, T=T, s=s, seed=seed, pos=pos)

    def w_len(rng, u, v):
        return 1.0 / np.linalg.norm(pos[u] - pos[v], axis=1)

    return wl, UpdateStream(wl, r["updates"], ("hops", 2, 4), w_len)


def make_rmat(scale: int = 22, n_edges: int = 64_000_000, seed: int = 0, K: float = 100.0,
              T: int = 100, s: int = 32) -> tuple[Workload, UpdateStream]:
    """Power-law social-like graph: symmetrised R-MAT, unit weights; insertions
    between uniform random vertex pairs.

    Drawing the scale-22 graph takes about a minute; when the environment
    variable DG_WORKLOAD_CACHE names a directory, the graph and H(0) are kept
    there (one .npz per scale, edge count and seed) and read back by later
    calls.  The update stream has its own generator, so it is the same either
    way."""
    r = rngs(seed)
    cache = os.environ.get("DG_WORKLOAD_CACHE")
    path = os.path.join(cache, f"rmat_v2_s{scale}_m{n_edges}_seed{seed}.npz") if cache else None
    if path and os.path.exists(path):
        with np.load(path) as z:
            n, a, b, h = int(z["n"]), z["a"], z["b"], z["h"]
    else:
        n, a, b = rmat(scale, n_edges, r["structure"])
        h = init_sparsifier(n, a, b, np.ones(a.size), r["init_h"])
        if path:
            os.makedirs(cache, exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp.npz"
            np.savez(tmp, n=n, a=a, b=b, h=h)
            os.replace(tmp, path)
    w = np.ones(a.size)
    wl = Workload(f"rmat_s{scale}", n, a, b, w, h, K=K, T=T, s=s, seed=seed)
    return wl, UpdateStream(wl, r["updates"], ("uniform",), lambda rng, u, v: np.ones(len(u)))


def serving_arrivals(n_requests: int, rate_per_s: float, rng: np.random.Generator,
                     max_batch: int = 50_000):
    """Poisson arrival times and log-uniform batch sizes floor(exp(U(0, ln(max+1))))."""
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps)
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(max_batch + 1), size=n_requests))).astype(np.int64)
    sizes = np.clip(sizes, 1, max_batch)
    return t, sizes
