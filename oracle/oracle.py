"""ctypes shim over the plain C oracle (dg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline / reference arm; the product path never loads it.

``build()`` compiles ``dg_oracle.c`` with ``gcc -O2 -ffp-contract=off`` so that
every FP64 add and multiply is rounded on its own, as the paper's estimator is
written (Eq. 12: sums of r_e in walk order; threshold w_pq * R > K).  It builds
the file twice: ``libdg_oracle.so`` (single-threaded) and, with ``-fopenmp``,
``libdg_oracle_omp.so``, whose walk phase runs the updates of a batch on
several host threads (the multi-threaded CPU form of Section III-E/F) with
identical results.  ``OracleGraph(threads=k)`` selects the second.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dg_oracle.c")
LIB = os.path.join(HERE, "libdg_oracle.so")
LIB_OMP = os.path.join(HERE, "libdg_oracle_omp.so")

# walker stop reasons (dg_oracle.c)
STOP_HIT, STOP_OVER_K, STOP_AT_T, STOP_LEAF, STOP_CUT = 1, 2, 3, 4, 5

WALKER_DTYPE = np.dtype([("reason", "<i4"), ("steps", "<i4"), ("R", "<f8")])


def _compile(out: str, extra: list) -> None:
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unknown-pragmas", *extra, "-o", out + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile the oracle (both builds) into shared libraries next to its source."""
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            _compile(out, extra)
    return LIB


_libs = {}


def lib(omp: bool = False):
    """The single-threaded oracle library, or its OpenMP build (omp=True)."""
    if omp not in _libs:
        build()
        L = C.CDLL(LIB_OMP if omp else LIB)
        P = C.c_void_p
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_create.argtypes = [C.c_int32, C.c_int64, i32p, i32p, f64p, C.c_uint64, C.c_double,
                                 C.c_int32, C.c_int32, C.c_int32]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_destroy.restype = None
        L.orc_init_sparsifier.argtypes = [P, C.c_int64, i32p, i32p]
        L.orc_init_sparsifier.restype = C.c_int
        L.orc_walk.argtypes = [P, C.c_int, C.c_int32, C.c_int32, C.c_double, C.c_int, C.c_uint64,
                               C.c_uint32, C.POINTER(C.c_int32), C.POINTER(C.c_double), P]
        L.orc_walk.restype = C.c_int
        L.orc_apply_batch.argtypes = [P, C.c_int64, i32p, i32p, f64p, i32p, i32p, u8p, u8p, u8p, u8p,
                                      i32p, i32p, i32p, i32p, f64p, P, P, P, P, P, P]
        L.orc_apply_batch.restype = C.c_int
        L.orc_query.argtypes = [P, C.c_int, C.c_int64, i32p, i32p, f64p]
        L.orc_query.restype = C.c_int64
        L.orc_degree.argtypes = [P, C.c_int, C.c_int32]
        L.orc_degree.restype = C.c_int32
        L.orc_next_id.argtypes = [P]
        L.orc_next_id.restype = C.c_uint64
        L.orc_set_next_id.argtypes = [P, C.c_uint64]
        L.orc_set_next_id.restype = None
        L.orc_tree_stretch.argtypes = [C.c_int32, C.c_int64, i32p, i32p, f64p, u8p, f64p]
        L.orc_tree_stretch.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_set_threads.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = C.c_int32
        _libs[omp] = L
    return _libs[omp]


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for one 128-bit counter and 64-bit key."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32),
                            out)
    return out


def tree_stretch(n, a, b, w, tree_ids):
    """Stretch w_e * R_T(e) of every edge of G (canonical arrays a, b, w) with
    respect to the spanning forest given by the edge ids tree_ids (0 for the
    tree edges, +inf across trees); raises if those edges hold a cycle."""
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    mask = np.zeros(a.size, np.uint8)
    mask[np.asarray(tree_ids, np.int64)] = 1
    out = np.zeros(a.size, np.float64)
    rc = lib().orc_tree_stretch(int(n), a.size, a, b, w, mask, out)
    if rc == -1:
        raise ValueError("the tree edges contain a cycle or a bad vertex")
    if rc != 0:
        raise MemoryError("oracle stretch failed")
    return out


def grass_sparsifier(n, a, b, w, tree_ids, n_off):
    """H(0) of the GRASS-like rule: the spanning forest plus the n_off off-tree
    edges of largest stretch (ties: smaller edge id); returns sorted edge ids."""
    st = tree_stretch(n, a, b, w, tree_ids)
    tree = np.zeros(a.size, bool)
    tree[np.asarray(tree_ids, np.int64)] = True
    off = np.nonzero(~tree)[0]
    order = np.lexsort((off, -st[off]))  # stretch descending, then id ascending
    pick = off[order[: int(n_off)]]
    return np.sort(np.concatenate([np.nonzero(tree)[0], pick]))


class OracleGraph:
    """One dynamic graph G with its sparsifier H, driven update by update."""

    def __init__(self, n, u, v, w, *, seed=0, K=100.0, T=100, s=32, early_exit=True, threads=1):
        """threads > 1 (or 0 = every host core) uses the OpenMP build."""
        self.n, self.T, self.s = int(n), int(T), int(s)
        self._lib = lib(omp=threads != 1)
        if threads != 1:
            self._lib.orc_set_threads(int(threads) if threads > 0 else (os.cpu_count() or 1))
        self.threads = int(self._lib.orc_max_threads())
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        w = np.ascontiguousarray(w, np.float64)
        self._h = self._lib.orc_create(self.n, u.size, u, v, w, int(seed), float(K), self.T, self.s,
                                   1 if early_exit else 0)
        if not self._h:
            raise ValueError("oracle rejected the graph (not simple, ids out of range or bad weight)")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init_sparsifier(self, hu, hv):
        rc = self._lib.orc_init_sparsifier(self._h, len(hu), np.ascontiguousarray(hu, np.int32),
                                       np.ascontiguousarray(hv, np.int32))
        if rc != 0:
            raise ValueError("oracle rejected the sparsifier (edge not in G)")

    @property
    def next_id(self) -> int:
        return int(self._lib.orc_next_id(self._h))

    @next_id.setter
    def next_id(self, value: int):
        self._lib.orc_set_next_id(self._h, int(value))

    def walk(self, p, q, wpq, deletion, upd_id, walker, on_h=True):
        """One walker; returns (reason, steps, R, path)."""
        steps = C.c_int32()
        R = C.c_double()
        path = np.full(self.T + 1, -1, np.int32)
        reason = self._lib.orc_walk(self._h, 1 if on_h else 0, int(p), int(q), float(wpq),
                                1 if deletion else 0, int(upd_id), int(walker), C.byref(steps),
                                C.byref(R), path.ctypes.data)
        if reason < 0:
            raise ValueError("vertex out of range")
        return reason, steps.value, R.value, path[: steps.value + 1].copy()

    def apply(self, u, v, w, op, *, walkers=False, paths=False, walk_mask=None, prune_bounds=False):
        """Apply one batch; returns a dict of per-update arrays (and walker records).

        walk_mask (optional bool array): walk only the marked updates (sampling
        mode for very large batches; H then lacks the unsampled commits).
        prune_bounds: also return nhits_min and steps_lo, the values nhits and
        steps take for a walked deletion whose walkers stop once their
        resistance exceeds R~ (equal to nhits and steps elsewhere), and with
        walkers=True every walker's record under that cut ("walkers_lo")."""
        mask = None if walk_mask is None else np.ascontiguousarray(walk_mask, np.uint8)
        nu = len(u)
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        w = np.ascontiguousarray(w, np.float64)
        op = np.ascontiguousarray(op, np.int32)
        out = dict(status=np.zeros(nu, np.int32), walked=np.zeros(nu, np.uint8),
                   hit=np.zeros(nu, np.uint8), accepted=np.zeros(nu, np.uint8),
                   fallback=np.zeros(nu, np.uint8), nhits=np.zeros(nu, np.int32),
                   best_walker=np.zeros(nu, np.int32), nrecovered=np.zeros(nu, np.int32),
                   steps=np.zeros(nu, np.int32), r_est=np.zeros(nu, np.float64))
        if prune_bounds:
            out["nhits_min"] = np.zeros(nu, np.int32)
            out["steps_lo"] = np.zeros(nu, np.int32)
        wout = np.zeros(nu * self.s, WALKER_DTYPE) if walkers else None
        wlo = np.zeros(nu * self.s, WALKER_DTYPE) if walkers and prune_bounds else None
        pbuf = np.full(nu * self.s * (self.T + 1), -1, np.int32) if paths else None
        rc = self._lib.orc_apply_batch(self._h, nu, u, v, w, op, out["status"], out["walked"], out["hit"],
                                       out["accepted"], out["fallback"], out["nhits"], out["best_walker"],
                                       out["nrecovered"], out["steps"], out["r_est"],
                                       None if wout is None else wout.ctypes.data,
                                       None if pbuf is None else pbuf.ctypes.data,
                                       None if mask is None else mask.ctypes.data,
                                       out["nhits_min"].ctypes.data if prune_bounds else None,
                                       out["steps_lo"].ctypes.data if prune_bounds else None,
                                       None if wlo is None else wlo.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle batch failed")
        if walkers:
            out["walkers"] = wout.reshape(nu, self.s)
        if wlo is not None:
            out["walkers_lo"] = wlo.reshape(nu, self.s)
        if paths:
            out["paths"] = pbuf.reshape(nu, self.s, self.T + 1)
        return out

    def apply_sequential(self, u, v, w, op, *, prune_bounds=False):
        """The updates one at a time, as Algorithm 1 states it: each one a batch
        of its own, so every update sees the G and H all earlier ones left.
        Returns the per-update arrays of all of them."""
        outs = [self.apply(u[i:i + 1], v[i:i + 1], w[i:i + 1], op[i:i + 1], prune_bounds=prune_bounds)
                for i in range(len(u))]
        if not outs:
            return self.apply(u, v, w, op, prune_bounds=prune_bounds)
        return {k: np.concatenate([o[k] for o in outs]) for k in outs[0]}

    def edges(self, which="H"):
        """(a, b, w) of H or G, a < b, lexicographic."""
        wh = 1 if which == "H" else 0
        dummy_i = np.zeros(1, np.int32)
        dummy_f = np.zeros(1, np.float64)
        cnt = self._lib.orc_query(self._h, wh, 0, dummy_i, dummy_i, dummy_f)
        a = np.zeros(max(cnt, 1), np.int32)
        b = np.zeros(max(cnt, 1), np.int32)
        w = np.zeros(max(cnt, 1), np.float64)
        self._lib.orc_query(self._h, wh, cnt, a, b, w)
        return a[:cnt], b[:cnt], w[:cnt]

    def degree(self, x, which="H"):
        return int(self._lib.orc_degree(self._h, 1 if which == "H" else 0, int(x)))
