"""Python binding of libdygrass.so (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and statuses to exceptions.  PyTorch is used
for device memory (optional allocator hook, device-resident batches) and
streams.  The binding never falls back to anything else: if the library is
missing or no GPU is present, it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdygrass.so")

DG_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error", -4: "timeout",
          -5: "invalid state", -6: "busy"}
OP_INSERT, OP_DELETE = 0, 1
WALK_BATCHED, WALK_PER_UPDATE = 0, 1

UPDATE_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("w", "<f8"), ("op", "<i4"), ("reserved", "<i4")])
RESULT_DTYPE = np.dtype([("status", "<i4"), ("walked", "u1"), ("hit", "u1"), ("accepted", "u1"),
                         ("fallback", "u1"), ("nhits", "<i4"), ("best_walker", "<i4"), ("nrecovered", "<i4"),
                         ("steps", "<i4"), ("r_est", "<f8")])
assert UPDATE_DTYPE.itemsize == 24 and RESULT_DTYPE.itemsize == 32
QUERY_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("w", "<f8"), ("kind", "<i4"), ("reserved", "<i4"),
                        ("id", "<u8")])
ESTIMATE_DTYPE = np.dtype([("status", "<i4"), ("nhits", "<i4"), ("best_walker", "<i4"), ("steps", "<i4"),
                           ("r_est", "<f8"), ("hit", "u1"), ("reserved", "u1", (7,))])
assert QUERY_DTYPE.itemsize == 32 and ESTIMATE_DTYPE.itemsize == 32
# one walked update's outcome exported by a shard of a sharded batch (ShardRec, 48 bytes)
SHARD_DTYPE = np.dtype([("j", "<u4"), ("best", "<i4"), ("best_steps", "<u4"), ("reserved", "<u4"),
                        ("result", RESULT_DTYPE)])
assert SHARD_DTYPE.itemsize == 48
NOALLOC_MAX_QUERIES = 4096
NOALLOC_MAX_WALKERS = 131072

# every symbol the header declares
EXPORTS = ("dg_config_default", "dg_create", "dg_destroy", "dg_status_str", "dg_last_error", "dg_load_graph",
           "dg_unload_graph", "dg_init_sparsifier", "dg_apply_updates", "dg_apply_updates_device",
           "dg_query_sparsifier", "dg_query_graph", "dg_get_batch_stats", "dg_get_walker_records", "dg_compact",
           "dg_graph_bytes", "dg_launch_count", "dg_set_next_update_id", "dg_get_next_update_id",
           "dg_set_walk_shape", "dg_set_walk_refill", "dg_submit_updates", "dg_wait", "dg_walk_estimate_noalloc",
           "dg_debug_set_wait_limit", "dg_shard_begin", "dg_shard_export", "dg_shard_commit", "dg_wait_ex",
           "dg_prepare", "dg_init_sparsifier_grass", "dg_sparsifier_density", "dg_laplacian_apply",
           "dg_pcg_solve", "dg_condition_number", "dg_debug_sparsifier_forest", "dg_debug_forest_solve",
           "dg_apply_updates_sequential", "dg_set_walk_coop", "dg_get_tune_log")

LAP_G, LAP_H = 0, 1
PRECOND = {"none": 0, "jacobi": 1, "sparsifier": 2}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("K", C.c_double), ("T", C.c_int32), ("s", C.c_int32),
                ("ins_early_exit", C.c_int32), ("del_prune", C.c_int32), ("walk_mode", C.c_int32),
                ("slack", C.c_double),
                ("overflow_frac", C.c_double), ("hbm_budget_bytes", C.c_uint64), ("autotune", C.c_int32),
                ("timeout_ms", C.c_int32), ("use_cuda_graphs", C.c_int32), ("record_walkers", C.c_int32),
                ("device", C.c_int32), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class BatchStats(C.Structure):
    _fields_ = [("updates", C.c_int64), ("valid", C.c_int64), ("walked", C.c_int64), ("steps", C.c_int64),
                ("accepted", C.c_int64), ("recovered", C.c_int64), ("h_edges", C.c_int64),
                ("g_edges", C.c_int64), ("walk_ms", C.c_double), ("batch_ms", C.c_double),
                ("walk_launches", C.c_int64), ("launches", C.c_int64), ("retries", C.c_int64),
                ("walk_block", C.c_int32), ("walk_ilp", C.c_int32), ("walk_blocks_per_sm", C.c_int32),
                ("graph_replayed", C.c_int32), ("mutate_ms", C.c_double), ("reduce_ms", C.c_double),
                ("emit_ms", C.c_double), ("commit_ms", C.c_double), ("walk_cut", C.c_int32),
                ("autotuned", C.c_int32), ("walk_refill", C.c_int32), ("walk_lanes", C.c_int32),
                ("walk_tile", C.c_int32), ("reserved0", C.c_int32), ("merge_ms", C.c_double),
                ("merge_entries", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PcgOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precond", C.c_int32), ("inner_tol", C.c_double),
                ("inner_max_iter", C.c_int32), ("reserved", C.c_int32)]


class PcgInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("inner_iters", C.c_int64), ("inner_max", C.c_int32), ("inner_unconverged", C.c_int32),
                ("ms", C.c_double)]


class KappaOptions(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("check_every", C.c_int32), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("inner_max_iter", C.c_int32), ("reserved", C.c_int32), ("d_v0", C.c_void_p), ("seed", C.c_uint64)]


class KappaInfo(C.Structure):
    _fields_ = [("kappa", C.c_double), ("lambda_min", C.c_double), ("iters", C.c_int32), ("converged", C.c_int32),
                ("inner_iters", C.c_int64), ("ms", C.c_double)]


def _as_dict(st):
    return {k: getattr(st, k) for k, _ in st._fields_ if not k.startswith("reserved")}


class DgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str | None = None):
    """Load libdygrass.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} is missing: build it with `python -m paper_2505_02741_b300.build`")
    L = C.CDLL(p)
    P, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "dg_config_default": (None, [C.POINTER(Config)]),
        "dg_create": (i32, [C.POINTER(Config), C.POINTER(P)]),
        "dg_destroy": (i32, [P]),
        "dg_status_str": (C.c_char_p, [i32]),
        "dg_last_error": (C.c_char_p, []),
        "dg_load_graph": (i32, [P, i32, i64, P, P, P, C.POINTER(i32)]),
        "dg_unload_graph": (i32, [P, i32]),
        "dg_init_sparsifier": (i32, [P, i32, i64, P, P]),
        "dg_apply_updates": (i32, [P, i32, i64, P, P, P]),
        "dg_apply_updates_device": (i32, [P, i32, i64, P, P, P]),
        "dg_query_sparsifier": (i32, [P, i32, i64, P, P, P, C.POINTER(i64)]),
        "dg_query_graph": (i32, [P, i32, i64, P, P, P, C.POINTER(i64)]),
        "dg_get_batch_stats": (i32, [P, i32, C.POINTER(BatchStats)]),
        "dg_get_walker_records": (i32, [P, i32, i64, P, P, P]),
        "dg_compact": (i32, [P, i32]),
        "dg_graph_bytes": (i32, [P, i32, C.POINTER(u64)]),
        "dg_launch_count": (u64, [P]),
        "dg_set_next_update_id": (i32, [P, i32, u64]),
        "dg_get_next_update_id": (i32, [P, i32, C.POINTER(u64)]),
        "dg_set_walk_shape": (i32, [P, i32, i32, i32, i32]),
        "dg_set_walk_refill": (i32, [P, i32, i32]),
        "dg_submit_updates": (i32, [P, i32, i64, P, P, C.POINTER(u64)]),
        "dg_wait": (i32, [P, u64, i32, C.POINTER(C.c_double)]),
        "dg_walk_estimate_noalloc": (i32, [P, i32, i64, P, P, P]),
        "dg_debug_set_wait_limit": (i32, [P, i64]),
        "dg_shard_begin": (i32, [P, i32, i64, P, i32, i32, P, C.POINTER(u64)]),
        "dg_shard_export": (i32, [P, i32, P, u64, C.POINTER(u64)]),
        "dg_shard_commit": (i32, [P, i32, u64, P, P]),
        "dg_wait_ex": (i32, [P, u64, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "dg_prepare": (i32, [P, i32, i64]),
        "dg_init_sparsifier_grass": (i32, [P, i32, i64, P, P, i64, P]),
        "dg_sparsifier_density": (i32, [P, i32, C.POINTER(C.c_double), C.POINTER(i64), C.POINTER(i64)]),
        "dg_laplacian_apply": (i32, [P, i32, i32, P, P, P]),
        "dg_pcg_solve": (i32, [P, i32, P, P, C.POINTER(PcgOptions), C.POINTER(PcgInfo), P]),
        "dg_condition_number": (i32, [P, i32, C.POINTER(KappaOptions), C.POINTER(KappaInfo)]),
        "dg_debug_sparsifier_forest": (i32, [P, i32, i64, P, P, C.POINTER(i64)]),
        "dg_debug_forest_solve": (i32, [P, i32, P, P]),
        "dg_apply_updates_sequential": (i32, [P, i32, i64, P, P, C.POINTER(i64)]),
        "dg_set_walk_coop": (i32, [P, i32, i32, i32]),
        "dg_get_tune_log": (i32, [P, i32, i64, P, P, C.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(rc):
    if rc != DG_OK:
        msg = _lib.dg_last_error().decode(errors="replace") if _lib else ""
        raise DgError(rc, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_updates(u, v, w, op) -> np.ndarray:
    """Pack arrays into the 24-byte dg_update records."""
    ups = np.zeros(len(u), UPDATE_DTYPE)
    ups["u"] = u
    ups["v"] = v
    ups["w"] = w
    ups["op"] = op
    return ups


class Context:
    def __init__(self, *, seed=0, K=100.0, T=100, s=32, early_exit=True, del_prune=True, walk_mode="batched",
                 slack=1.25, overflow=0.5, hbm_budget=0, autotune=True, timeout_ms=60000, cuda_graphs=True,
                 record_walkers=False, device=0, allocator=None):
        L = load_library()
        cfg = Config()
        L.dg_config_default(C.byref(cfg))
        cfg.seed, cfg.K, cfg.T, cfg.s = int(seed), float(K), int(T), int(s)
        cfg.ins_early_exit = 1 if early_exit else 0
        cfg.del_prune = 1 if del_prune else 0
        cfg.walk_mode = WALK_PER_UPDATE if walk_mode in ("per_update", WALK_PER_UPDATE) else WALK_BATCHED
        cfg.slack, cfg.overflow_frac = float(slack), float(overflow)
        cfg.hbm_budget_bytes = int(hbm_budget)
        cfg.autotune = 1 if autotune else 0
        cfg.timeout_ms = int(timeout_ms)
        cfg.use_cuda_graphs = 1 if cuda_graphs else 0
        cfg.record_walkers = 1 if record_walkers else 0
        cfg.device = int(device)
        self._hooks = None
        if allocator == "torch":
            import torch

            dev = int(device)

            def _alloc(nbytes, stream, user):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
            cfg.alloc, cfg.free = self._hooks
        self.T, self.s = int(T), int(s)
        self.del_prune = bool(del_prune)
        h = C.c_void_p()
        _check(L.dg_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._lib = L

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.dg_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(self._lib.dg_launch_count(self._h))

    def debug_set_wait_limit(self, polls: int):
        """Polls of the walk's finalize-queue wait before it gives up (< 0: default)."""
        _check(self._lib.dg_debug_set_wait_limit(self._h, int(polls)))

    def load_graph(self, n, u, v, w) -> "Graph":
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        w = np.ascontiguousarray(w, np.float64)
        gid = C.c_int32()
        _check(self._lib.dg_load_graph(self._h, int(n), u.size, _ptr(u), _ptr(v), _ptr(w), C.byref(gid)))
        return Graph(self, gid.value, int(n))

    def wait(self, ticket, timeout_ms=-1):
        lat = C.c_double()
        rc = self._lib.dg_wait(self._h, int(ticket), int(timeout_ms), C.byref(lat))
        _check(rc)
        return lat.value

    def wait_ex(self, ticket, timeout_ms=-1):
        """(latency_ms, queue_ms) of a served request."""
        lat, q = C.c_double(), C.c_double()
        _check(self._lib.dg_wait_ex(self._h, int(ticket), int(timeout_ms), C.byref(lat), C.byref(q)))
        return lat.value, q.value


class Graph:
    def __init__(self, ctx: Context, gid: int, n: int):
        self.ctx, self.gid, self.n = ctx, gid, n
        self._L = ctx._lib
        self._keep = {}

    def unload(self):
        _check(self._L.dg_unload_graph(self.ctx._h, self.gid))

    def init_sparsifier(self, u, v):
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        _check(self._L.dg_init_sparsifier(self.ctx._h, self.gid, u.size, _ptr(u), _ptr(v)))

    def init_sparsifier_grass(self, tree_u, tree_v, n_off: int, with_stretch=False):
        """GRASS-like H(0): the forest (tree_u, tree_v) plus the n_off off-tree
        edges of largest stretch; optionally returns every edge's stretch
        (lexicographic edge order)."""
        tu = np.ascontiguousarray(tree_u, np.int32)
        tv = np.ascontiguousarray(tree_v, np.int32)
        out = None
        if with_stretch:
            cnt = C.c_int64()
            _check(self._L.dg_query_graph(self.ctx._h, self.gid, 0, None, None, None, C.byref(cnt)))
            out = np.zeros(max(cnt.value, 1), np.float64)
        _check(self._L.dg_init_sparsifier_grass(self.ctx._h, self.gid, tu.size, _ptr(tu), _ptr(tv), int(n_off),
                                                _ptr(out)))
        return None if out is None else out[: cnt.value]

    def apply(self, ups: np.ndarray, stream=None, out: np.ndarray | None = None) -> np.ndarray:
        """One batch from host records; returns the result records (into ``out``
        when given: a RESULT_DTYPE array of at least ups.size records).  With
        pinned arrays (e.g. numpy views of pinned torch tensors) the library
        copies them directly instead of staging them."""
        ups = np.ascontiguousarray(ups, UPDATE_DTYPE)
        if out is None:
            res = np.zeros(ups.size, RESULT_DTYPE)
        else:
            if out.dtype != RESULT_DTYPE or out.size < ups.size or not out.flags.c_contiguous:
                raise ValueError("out must be a contiguous RESULT_DTYPE array with room for every update")
            res = out[: ups.size]
        _check(self._L.dg_apply_updates(self.ctx._h, self.gid, ups.size, _ptr(ups), _ptr(res),
                                        None if stream is None else C.c_void_p(int(stream))))
        return res

    def apply_device(self, d_ups_ptr: int, nu: int, d_res_ptr: int | None, stream=None):
        """One batch whose records already live in device memory (e.g. torch tensors)."""
        _check(self._L.dg_apply_updates_device(self.ctx._h, self.gid, int(nu), C.c_void_p(int(d_ups_ptr)),
                                               None if not d_res_ptr else C.c_void_p(int(d_res_ptr)),
                                               None if stream is None else C.c_void_p(int(stream))))

    def _query(self, fn):
        cnt = C.c_int64()
        _check(fn(self.ctx._h, self.gid, 0, None, None, None, C.byref(cnt)))
        n = cnt.value
        a = np.zeros(max(n, 1), np.int32)
        b = np.zeros(max(n, 1), np.int32)
        w = np.zeros(max(n, 1), np.float64)
        _check(fn(self.ctx._h, self.gid, n, _ptr(a), _ptr(b), _ptr(w), C.byref(cnt)))
        return a[:n], b[:n], w[:n]

    def sparsifier(self):
        """(u, v, w) of H, u < v, lexicographic."""
        return self._query(self._L.dg_query_sparsifier)

    def edges(self):
        """(u, v, w) of the current G."""
        return self._query(self._L.dg_query_graph)

    def stats(self) -> dict:
        st = BatchStats()
        _check(self._L.dg_get_batch_stats(self.ctx._h, self.gid, C.byref(st)))
        return st.as_dict()

    def walker_records(self, nu: int, paths=True):
        rows = nu * self.ctx.s
        reason = np.zeros(rows, np.int32)
        steps = np.zeros(rows, np.int32)
        pbuf = np.full(rows * (self.ctx.T + 1), -1, np.int32) if paths else None
        _check(self._L.dg_get_walker_records(self.ctx._h, self.gid, nu, _ptr(reason), _ptr(steps), _ptr(pbuf)))
        out = dict(reason=reason.reshape(nu, self.ctx.s), steps=steps.reshape(nu, self.ctx.s))
        if paths:
            out["paths"] = pbuf.reshape(nu, self.ctx.s, self.ctx.T + 1)
        return out

    def compact(self):
        _check(self._L.dg_compact(self.ctx._h, self.gid))

    def device_bytes(self) -> int:
        b = C.c_uint64()
        _check(self._L.dg_graph_bytes(self.ctx._h, self.gid, C.byref(b)))
        return b.value

    @property
    def next_update_id(self) -> int:
        x = C.c_uint64()
        _check(self._L.dg_get_next_update_id(self.ctx._h, self.gid, C.byref(x)))
        return x.value

    @next_update_id.setter
    def next_update_id(self, value: int):
        _check(self._L.dg_set_next_update_id(self.ctx._h, self.gid, int(value)))

    def set_walk_shape(self, block=0, ilp=0, blocks_per_sm=0, refill=0):
        _check(self._L.dg_set_walk_shape(self.ctx._h, self.gid, int(block), int(ilp), int(blocks_per_sm)))
        if refill:
            _check(self._L.dg_set_walk_refill(self.ctx._h, self.gid, int(refill)))

    def set_walk_coop(self, lanes=1, tile=0):
        """Lanes per walker and the frontier tile (updates per block claim; 0 = walker queue)."""
        _check(self._L.dg_set_walk_coop(self.ctx._h, self.gid, int(lanes), int(tile)))

    def tune_log(self):
        """The autotuner's trials: list of (shape dict, median walk ms)."""
        cnt = C.c_int64()
        cap = 256
        shapes = np.zeros(6 * cap, np.int32)
        ms = np.zeros(cap, np.float32)
        _check(self._L.dg_get_tune_log(self.ctx._h, self.gid, cap, _ptr(shapes), _ptr(ms), C.byref(cnt)))
        keys = ("block", "ilp", "refill", "lanes", "tile", "cut")
        return [(dict(zip(keys, shapes[6 * i:6 * i + 6].tolist())), float(ms[i])) for i in range(cnt.value)]

    def walk_estimate_noalloc(self, d_queries_ptr: int, nq: int, d_out_ptr: int, stream=None):
        """Walk estimates for nq device-resident queries; the call allocates no
        device memory (its scratch is a fixed static array in the library) and
        returns once the work is enqueued on ``stream``."""
        _check(self._L.dg_walk_estimate_noalloc(self.ctx._h, self.gid, int(nq), C.c_void_p(int(d_queries_ptr)),
                                                C.c_void_p(int(d_out_ptr)),
                                                None if stream is None else C.c_void_p(int(stream))))

    def shard_begin(self, ups: np.ndarray, rank: int, world: int, stream=None) -> int:
        """Sharded batch, step 1: mutate, walk this replica's share; returns its record count."""
        ups = np.ascontiguousarray(ups, UPDATE_DTYPE)
        n = C.c_uint64()
        _check(self._L.dg_shard_begin(self.ctx._h, self.gid, ups.size, _ptr(ups), int(rank), int(world),
                                      None if stream is None else C.c_void_p(int(stream)), C.byref(n)))
        self._shard_nu = ups.size
        return n.value

    def shard_export(self) -> np.ndarray:
        """Sharded batch, step 2: this replica's records (SHARD_DTYPE)."""
        n = C.c_uint64()
        _check(self._L.dg_shard_export(self.ctx._h, self.gid, None, 0, C.byref(n)))
        recs = np.zeros(n.value, SHARD_DTYPE)
        _check(self._L.dg_shard_export(self.ctx._h, self.gid, _ptr(recs), recs.size, C.byref(n)))
        return recs

    def shard_commit(self, recs: np.ndarray) -> np.ndarray:
        """Sharded batch, step 3: every replica's records (concatenated, any
        order); commits the batch and returns every update's result."""
        recs = np.ascontiguousarray(recs, SHARD_DTYPE)
        res = np.zeros(self._shard_nu, RESULT_DTYPE)
        _check(self._L.dg_shard_commit(self.ctx._h, self.gid, recs.size, _ptr(recs), _ptr(res)))
        return res

    def apply_sharded(self, ups: np.ndarray, rank: int, world: int, gather) -> np.ndarray:
        """One batch as shard `rank` of `world`: ``gather(records)`` must return
        the records of every shard (e.g. ``shard.allgather_records``)."""
        self.shard_begin(ups, rank, world)
        return self.shard_commit(gather(self.shard_export()))

    def submit(self, ups: np.ndarray):
        """Queue one request; returns (ticket, result array filled when waited)."""
        ups = np.ascontiguousarray(ups, UPDATE_DTYPE)
        res = np.zeros(ups.size, RESULT_DTYPE)
        t = C.c_uint64()
        _check(self._L.dg_submit_updates(self.ctx._h, self.gid, ups.size, _ptr(ups), _ptr(res), C.byref(t)))
        self._keep[t.value] = (ups, res)
        return t.value, res

    def wait(self, ticket, timeout_ms=-1):
        lat = self.ctx.wait(ticket, timeout_ms)
        ups, res = self._keep.pop(ticket)
        return res, lat

    def wait_ex(self, ticket, timeout_ms=-1):
        """(results, latency_ms, queue_ms) of a served request."""
        lat, q = self.ctx.wait_ex(ticket, timeout_ms)
        ups, res = self._keep.pop(ticket)
        return res, lat, q

    def prepare(self, max_batch: int):
        """Size the workspace and capture the batch steps for batches up to max_batch."""
        _check(self._L.dg_prepare(self.ctx._h, self.gid, int(max_batch)))

    def apply_sequential(self, ups: np.ndarray):
        """The updates one at a time (Algorithm 1's order; every update sees all
        earlier ones).  Returns (results, number of batches it took)."""
        ups = np.ascontiguousarray(ups, UPDATE_DTYPE)
        res = np.zeros(ups.size, RESULT_DTYPE)
        pre = C.c_int64()
        _check(self._L.dg_apply_updates_sequential(self.ctx._h, self.gid, ups.size, _ptr(ups), _ptr(res),
                                                   C.byref(pre)))
        return res, pre.value

    # ---- quality of the sparsifier (Section IV) ------------------------------
    def density(self):
        """(d_H, |E(G)|, |E(H)|) with d_H = |E(H)| / |V| - 1."""
        d, mg, mh = C.c_double(), C.c_int64(), C.c_int64()
        _check(self._L.dg_sparsifier_density(self.ctx._h, self.gid, C.byref(d), C.byref(mg), C.byref(mh)))
        return d.value, mg.value, mh.value

    def laplacian_apply(self, which: int, d_x: int, d_y: int, stream=None):
        """y = L x for G (LAP_G) or H (LAP_H); device pointers to n doubles."""
        _check(self._L.dg_laplacian_apply(self.ctx._h, self.gid, int(which), d_x, d_y, stream))

    def pcg_solve(self, d_b: int, d_x: int, *, tol=1e-8, max_iter=1000, precond="sparsifier", inner_tol=1e-12,
                  inner_max_iter=5000, history=True):
        """PCG on L_G x = b (device pointers); returns (info dict, relative residual history)."""
        o = PcgOptions(tol=tol, max_iter=int(max_iter), precond=PRECOND[precond], inner_tol=inner_tol,
                       inner_max_iter=int(inner_max_iter))
        info = PcgInfo()
        hist = np.zeros(int(max_iter) + 1) if history else None
        _check(self._L.dg_pcg_solve(self.ctx._h, self.gid, d_b, d_x, C.byref(o), C.byref(info),
                                    _ptr(hist) if hist is not None else None))
        d = _as_dict(info)
        return d, (hist[: d["iters"] + 1] if hist is not None else None)

    def condition_number(self, *, max_iter=200, check_every=5, tol=1e-10, inner_tol=1e-12, inner_max_iter=5000,
                         d_v0=None, seed=0):
        """kappa(L_G, L_H) by Lanczos on the pencil; d_v0: device pointer to a start vector (or None)."""
        o = KappaOptions(max_iter=int(max_iter), check_every=int(check_every), tol=tol, inner_tol=inner_tol,
                         inner_max_iter=int(inner_max_iter), d_v0=d_v0, seed=int(seed))
        info = KappaInfo()
        _check(self._L.dg_condition_number(self.ctx._h, self.gid, C.byref(o), C.byref(info)))
        return _as_dict(info)

    def debug_sparsifier_forest(self):
        """Edges (u < v, lexicographic) of H's maximum-weight spanning forest."""
        nf = C.c_int64()
        fu = np.empty(max(self.n, 1), np.int32)
        fv = np.empty(max(self.n, 1), np.int32)
        _check(self._L.dg_debug_sparsifier_forest(self.ctx._h, self.gid, fu.size, _ptr(fu), _ptr(fv), C.byref(nf)))
        return fu[: nf.value].copy(), fv[: nf.value].copy()

    def debug_forest_solve(self, d_r: int, d_z: int):
        """z = L_F^+ r up to a constant per tree (z = 0 at each tree's smallest vertex)."""
        _check(self._L.dg_debug_forest_solve(self.ctx._h, self.gid, d_r, d_z))
