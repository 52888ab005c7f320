"""Benchmark: batched dyGRASS updates on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload rmat|mesh|fea|serve]

Default workload (the largest single-GPU configuration): symmetrised R-MAT
scale 22 (4.2M vertices, 64M undirected edges, a,b,c,d = .57,.19,.19,.05, unit
weights), H(0) = max-weight spanning forest + 10 % of the off-tree edges,
K = 100, T = 100, s = 32.  One step = one batch of 50k updates: 30k insertions
between random vertex pairs and 20k deletions of current edges, shuffled.  The
configuration's stream is 20 such batches from G(0); timed step k applies
batch k mod 20, every pass of the stream on a fresh copy of G(0) and H(0)
loaded outside the timed steps (the warm-up takes the stream's first W batches
on a copy of its own).
``--workload mesh`` (3-D mesh 100^3, 10k + 10k per batch) and ``fea`` (jittered
triangulated 2048^2 grid, 50k + 50k) are the other batch configurations;
``serve`` runs the serving configuration.  Synthetic data, seeded.

value    : updates/s of the batched form, batches already resident in HBM
           (dg_apply_updates_device), CUDA events on the batch stream, L2
           flushed (256 MB write) between steps.
e2e      : the same through dg_apply_updates with pinned host buffers (H2D of
           the batch, D2H of the results inside the timed region).
roofline : the walk kernel: algorithmic bytes = 20 B per useful walk step (the
           vertex record, the neighbour id and its resistance), against the
           measured HBM copy bandwidth; ``gather`` restates it at the sector
           level (two 32-byte sectors per step).
roofline_merge : the merge of G's touched lists (the largest kernel of the
           R-MAT step): 32 B per entry read from an old list or written to a
           new one, over the merge's CUDA-event time inside the step.
Also reported: walk-steps/s, the one-launch-per-update form at identical
outputs, the sequential semantics (every update sees all earlier ones,
Algorithm 1's order), per-batch latency p50/p99, and the CPU oracle on a
bounded sample of the same workload, single-threaded and on every host core.
``--workload quality`` runs Section IV's quality experiment (d_H, kappa and
PCG iterations with and without updates).

Under torchrun each rank runs an independent replica (its own seed); there is
no collective on the data path; rank 0 prints the whole-job line.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import platform
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the scale-22 graph takes about a minute to draw: keep it for the later runs on this host
os.environ.setdefault("DG_WORKLOAD_CACHE", "/tmp/dg_workload_cache")

METRIC = "updates/s & walk-steps/s on 1 B300, batched vs per-update; p50/p99 latency"
ALG_BYTES_PER_STEP = 20      # vertex record (8 B) + neighbour id (4 B) + its resistance (8 B)
SECTOR_BYTES_PER_STEP = 64   # the same step at DRAM-sector granularity (two 32-byte sectors)
# DRAM bytes (read + write) of one walk launch per workload, from one ncu
# capture of the current walk kernel (None while the kernel has changed since
# its last capture)
WALK_TRAFFIC = {
    "rmat": (2_231_460_000, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_walk_batched<1,1> launch, "
                            "R-MAT scale 22 default batch: 2.11 GB read + 121.5 MB written"),
    "mesh": (252_908_544, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_walk_batched<1,0> launch, "
                          "mesh 100^3, first timed batch: 226.9 MB read + 26.0 MB written"),
    "fea": (574_097_664, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_walk_batched<1,0> launch, "
                         "FEA 2048^2, first timed batch: 511.8 MB read + 62.3 MB written"),
}

# the list merge of G's mutation: one 32-byte entry read (old list) or written (new list)
MERGE_BYTES_PER_ENTRY = 32
MERGE_TRAFFIC = {
    "rmat": (2_840_000_000, "ncu dram__bytes_read.sum + dram__bytes_write.sum of G's k_exec_merge launch, "
                            "R-MAT scale 22 default batch: 1.46 GB read + 1.38 GB written"),
}

BATCH = {"rmat": (30_000, 20_000), "mesh": (10_000, 10_000), "fea": (50_000, 50_000)}
# batches in one pass of each configuration's update stream (R-MAT: 20 batches of
# 50k; mesh: 10 batches of 10k + 10k; FEA: 10 batches of 100k)
STREAM_BATCHES = {"rmat": 20, "mesh": 10, "fea": 10}


def make_workload(name, args, seed):
    from paper_2505_02741_b300 import workloads as W
    if name == "rmat":
        return W.make_rmat(scale=args.rmat_scale, n_edges=args.rmat_edges, seed=seed)
    if name == "fea":
        return W.make_fea(seed=seed)
    return W.make_mesh3d(seed=seed)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def host_cpu():
    model = platform.processor() or ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


class ClockSampler:
    """SM clocks and throttle reasons during the timed region.  One nvidia-smi
    process streams a sample every 20 ms (NVML every 5 ms where its Python
    binding loads), started before the warm-up so that its first samples are
    out by the time the region begins; the summary keeps the samples that
    arrived while a timed region ran (within one sampling interval of its end).
    The timed steps may form several regions (one per pass of the stream)."""

    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    QUERY = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD = 0.02

    def __init__(self, local=0):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.index = ids[local] if local < len(ids) else str(local)
        self.rows = []  # (host time, sm_mhz, max_mhz, set of active reasons)
        self.regions = []  # [start, end] host times of the timed regions
        self._stop = threading.Event()
        self._t = None
        self._proc = None
        self._nvml = None
        try:
            import pynvml as N
            N.nvmlInit()
            h = N.nvmlDeviceGetHandleByIndex(int(self.index)) if self.index.isdigit() else \
                N.nvmlDeviceGetHandleByUUID(self.index)
            self._nvml = (N, h)
        except Exception:
            self._nvml = None

    def _parse(self, line):
        r = [x.strip() for x in line.split(",")]
        if len(r) < 6 or not r[0].replace(".", "").isdigit():
            return None
        act = {n for n, x in zip(self.NAMES, r[2:]) if "Active" in x and "Not" not in x}
        return time.perf_counter(), float(r[0]), float(r[1]), act

    def _run_nvml(self):
        N, h = self._nvml
        masks = (0x8, 0x40, 0x20, 0x4)  # hw slowdown, hw thermal, sw thermal, sw power cap
        while not self._stop.is_set():
            try:
                bits = N.nvmlDeviceGetCurrentClocksThrottleReasons(h)
                self.rows.append((time.perf_counter(), float(N.nvmlDeviceGetClockInfo(h, N.NVML_CLOCK_SM)),
                                  float(N.nvmlDeviceGetMaxClockInfo(h, N.NVML_CLOCK_SM)),
                                  {n for n, m in zip(self.NAMES, masks) if bits & m}))
            except Exception:
                pass
            self._stop.wait(0.005)

    def _run_smi(self):
        for line in self._proc.stdout:
            row = self._parse(line)
            if row:
                self.rows.append(row)

    def start(self):
        if self._nvml:
            self._t = threading.Thread(target=self._run_nvml, daemon=True)
        else:
            cmd = ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                   "-lms", str(int(self.PERIOD * 1000))]
            if shutil.which("stdbuf"):
                cmd = ["stdbuf", "-oL"] + cmd  # each sample reaches the pipe when it is taken
            try:
                self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                                              bufsize=1)
                self._t = threading.Thread(target=self._run_smi, daemon=True)
            except OSError:
                self._proc = None
        if self._t:
            self._t.start()
        return self

    def begin(self):  # a timed region starts (there may be several)
        self.regions.append([time.perf_counter(), None])

    def end(self):
        self.regions[-1][1] = time.perf_counter()

    def __enter__(self):
        self.begin()
        return self

    def __exit__(self, *a):
        self.end()

    def stop(self):
        time.sleep(2 * self.PERIOD)  # the samples taken inside the last region reach the pipe
        self._stop.set()
        if self._proc:
            self._proc.terminate()  # the sampler process this object started
            try:
                self._proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        regs = [(a, b) for a, b in self.regions if b is not None]
        inside = [r for r in self.rows if any(a <= r[0] <= b + self.PERIOD for a, b in regs)]
        src = "nvml, 5 ms" if self._nvml else "nvidia-smi -lms 20"
        if not inside and regs:
            after = [r for r in self.rows if r[0] > regs[-1][1]]
            inside = after[:1]
            src += ", first sample after the region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(set().union(*(r[3] for r in inside))), "samples": len(inside), "source": src,
                "region_ms": 1e3 * sum(b - a for a, b in regs), "regions": len(regs)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(vals_sum, vals_max, world, backend):
    """Whole-job totals: sums of units, max of times (host-side, measurement only)."""
    if world == 1:
        return vals_sum, vals_max
    import torch
    import torch.distributed as dist
    dev = "cuda" if backend == "nccl" else "cpu"
    a = torch.tensor(vals_sum, dtype=torch.float64, device=dev)
    b = torch.tensor(vals_max, dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    return a.cpu().tolist(), b.cpu().tolist()


def stream_slices(batches, size):
    """The batch stream (any iterable of batches) cut into consecutive slices
    of `size` updates (each a valid batch in stream order)."""
    for bt in batches:
        for lo in range(0, len(bt), size):
            yield bt.u[lo:lo + size], bt.v[lo:lo + size], bt.w[lo:lo + size], bt.op[lo:lo + size]


def oracle_baseline(wl, batches, budget_s=12.0, slice_size=1000):
    """The CPU oracle on the stream from G(0): its walk phase on one host
    thread, then on every host core (its OpenMP build, identical outputs),
    each for about budget_s of work on consecutive slices of the stream.
    Returns (single-thread dict, all-core dict)."""
    from oracle.oracle import OracleGraph
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s, threads=0)
    cores = o.threads
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    it = stream_slices(batches, slice_size)
    out = []
    for threads in (1, cores):
        o._lib.orc_set_threads(threads)
        done, steps, t_tot, nsl = 0, 0, 0.0, 0
        for u, v, w, op in it:
            t0 = time.perf_counter()
            r = o.apply(u, v, w, op, prune_bounds=True)
            t_tot += time.perf_counter() - t0
            done += int((r["status"] == 0).sum())
            steps += int(r["steps_lo"].sum())
            nsl += 1
            if t_tot >= budget_s:
                break
        out.append({"value": done / t_tot, "unit": "updates/s", "cores": threads, "kind": "oracle",
                    "walk_steps_per_s": steps / t_tot, "seconds": t_tot,
                    "sample": f"{nsl} consecutive slices of {slice_size} updates of the stream from G(0)"})
    o.close()
    return out[0], out[1]


def run_reference(args):
    """--impl reference: the CPU oracle, single-threaded, on the same workload;
    each step a bounded sample (consecutive slices of the update stream)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.oracle import OracleGraph
    wl, st = make_workload(args.workload, args, 0)
    n_ins, n_del = BATCH[args.workload]
    sample = args.ref_sample
    nb = (args.warmup + args.steps) * sample // (n_ins + n_del) + 1
    batches = [st.next_batch(n_ins, n_del) for _ in range(nb)]
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    times, units = [], 0
    it = stream_slices(batches, sample)
    for i in range(args.warmup + args.steps):
        u, v, w, op = next(it)
        t0 = time.perf_counter()
        r = o.apply(u, v, w, op, prune_bounds=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            units += int((r["status"] == 0).sum())
    o.close()
    value = units / sum(times)
    samp = f"{args.steps} consecutive slices of {sample} updates of the stream, one host thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "batch": sample,
                                            "K": wl.K, "T": wl.T, "s": wl.s},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": samp,
                             **host_cpu()},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _split_requests(bt, sizes):
    """Cut one valid batch (distinct current-edge deletions, distinct new-edge
    insertions) into consecutive requests; each request stays valid in order."""
    out, lo = [], 0
    for s in sizes:
        out.append((bt.u[lo:lo + s], bt.v[lo:lo + s], bt.w[lo:lo + s], bt.op[lo:lo + s]))
        lo += s
    return out


SIZE_BUCKETS = ((1, 99), (100, 999), (1000, 9999), (10000, 50000))


def _pcts(x):
    x = np.asarray(x, np.float64)
    if x.size == 0:
        return None
    return {"n": int(x.size), "p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)),
            "max": float(x.max())}


def serve_experiment(loads, requests_per_point, seed=7, per_update_sample=6):
    """Serving: the 64x64 grid, the 100^3 mesh and the 2048^2 FEA-like mesh
    resident at once in one context.  Per graph a Poisson request stream,
    batch sizes floor(exp(U(0, ln 50001))) (at most 400 on the small grid),
    50/50 insertions/deletions.  Each graph's batched capacity is measured
    alone first; at offered load L every graph's stream runs at L x its
    capacity alone / 3 (the three share one GPU).  Before the measured
    streams every graph is prepared for requests of up to 50k updates (batch
    workspace sized, steps captured) and given the walk shape tuned alone.
    Per load point: updates/s, request latency (submit to results on the
    host) p50/p99 overall, per graph and per request-size bucket, and the
    part of it spent queued behind earlier requests of the same graph."""
    import torch
    from paper_2505_02741_b300 import dygrass as D
    from paper_2505_02741_b300 import workloads as W

    torch.cuda.init()
    specs = [("grid64", lambda: W.make_grid(64, 64, seed=0), 400),
             ("mesh100", lambda: W.make_mesh3d(seed=0), 50_000),
             ("fea2048", lambda: W.make_fea(seed=0), 50_000)]
    arr_rng = W.rngs(seed)["arrivals"]
    per_graph = max(4, requests_per_point // len(specs))
    graphs = []  # (name, wl, [requests of point 0], [point 1], ...)
    for name, mk, cap in specs:
        wl, st = mk()
        points = []
        for _ in range(len(loads) + 1):  # one stream per load point, plus one for the capacity runs
            _, sizes = W.serving_arrivals(per_graph, 1.0, arr_rng)
            sizes = np.minimum(sizes, cap)
            if name == "grid64":
                reqs = []
                for sz in sizes:
                    ins = int(sz) // 2
                    b = st.next_batch(ins, int(sz) - ins)
                    reqs.append((b.u, b.v, b.w, b.op))
            else:
                total = int(sizes.sum())
                big = st.next_batch(total // 2, total - total // 2)
                reqs = _split_requests(big, sizes)
            points.append(reqs)
        graphs.append((name, wl, points))

    def load(ctx, wl):
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        return g

    # batched capacity per graph alone, on its own copy (the first stream, sequential)
    cap_ups, shapes = {}, {}
    for name, wl, points in graphs:
        ctx = D.Context()
        g = load(ctx, wl)
        g.prepare(50_000)
        reqs = points[-1]
        big = max(range(len(reqs)), key=lambda k: len(reqs[k][0]))
        done, t_tot = 0, 0.0
        for k, r in enumerate(reqs):
            ups = D.make_updates(*r)
            t0 = time.perf_counter()
            g.apply(ups)
            dt = time.perf_counter() - t0
            if k >= 3 and k != big:  # warm-up requests and the autotuned one aside
                done += len(ups)
                t_tot += dt
        st_ = g.stats()
        shapes[name] = (st_["walk_block"], st_["walk_ilp"], st_["walk_refill"])
        cap_ups[name] = done / t_tot
        ctx.close()

    # the served streams, one load point after the other on the same resident graphs
    ctx = D.Context()
    gs = {}
    for name, wl, _ in graphs:
        g = load(ctx, wl)
        blk, ilp, refill = shapes[name]
        g.set_walk_shape(blk, ilp, 0, refill)
        g.prepare(50_000)
        gs[name] = g
    out = {"loads": {}, "capacity_updates_per_s": cap_ups,
           "graphs": {n: {"n": wl.n, "m": wl.m} for n, wl, _ in graphs}}
    for pi, lf in enumerate(loads):
        schedule = []
        for name, _, points in graphs:
            reqs = points[pi]
            mean = float(np.mean([len(r[0]) for r in reqs]))
            lam = lf * cap_ups[name] / len(graphs) / mean  # requests / s (the GPU is shared)
            t = np.cumsum(arr_rng.exponential(1.0 / lam, size=len(reqs)))
            for k, r in enumerate(reqs):
                schedule.append((float(t[k]), name, D.make_updates(*r)))
        schedule.sort(key=lambda x: x[0])
        tickets = []
        t_start = time.perf_counter()
        for at, name, ups in schedule:
            delay = at - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            tickets.append((name, len(ups)) + gs[name].submit(ups))
        rows, units = [], 0
        for name, nu, ticket, _res in tickets:
            res, ms, qms = gs[name].wait_ex(ticket, timeout_ms=600000)
            rows.append((name, nu, ms, qms))
            units += int((res["status"] == 0).sum())
        wall = time.perf_counter() - t_start
        lat = [r[2] for r in rows]
        point = {"requests": len(rows), "updates_per_s": units / wall, "offered_load": lf,
                 "latency_ms": _pcts(lat), "queue_ms": _pcts([r[3] for r in rows]),
                 "per_graph": {n: {"latency_ms": _pcts([r[2] for r in rows if r[0] == n]),
                                   "queue_ms": _pcts([r[3] for r in rows if r[0] == n])} for n in gs},
                 "per_size": {f"{lo}-{hi}": _pcts([r[2] for r in rows if lo <= r[1] <= hi])
                              for lo, hi in SIZE_BUCKETS}}
        out["loads"][str(lf)] = point
    ctx.close()

    # the one-launch-per-update form on a sample of the mesh requests (its first stream)
    name, wl, points = graphs[1]
    ctx = D.Context(walk_mode="per_update", cuda_graphs=False)
    g = load(ctx, wl)
    pu_lat, pu_units = [], 0
    for r in points[-1][:per_update_sample]:
        ups = D.make_updates(*r)
        t0 = time.perf_counter()
        res = g.apply(ups)
        pu_lat.append(1e3 * (time.perf_counter() - t0))
        pu_units += int((res["status"] == 0).sum())
    ctx.close()
    out["per_update_form"] = {"graph": "mesh100", "requests": len(pu_lat),
                              "updates_per_s": pu_units / (sum(pu_lat) / 1e3),
                              "latency_ms": _pcts(pu_lat)}
    return out


def run_serve(args):
    """--workload serve: the serving configuration at offered loads of 30, 60
    and 90 % of capacity, --requests per load point."""
    r = serve_experiment((0.3, 0.6, 0.9), args.requests)
    mid = r["loads"]["0.6"]
    line = {"metric": "serving: updates/s and p50/p99 request latency", "workload": "serve",
            "value": mid["updates_per_s"], "unit": "updates/s", "n_gpus": 1, "requests_per_point": args.requests,
            "offered_per_graph": "load x capacity alone / 3 (one GPU shared)",
            "latency_ms": mid["latency_ms"], "points": r, "dtype": "f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_quality(args):
    """--workload quality: the quality experiment of Section IV (Tables II-IV)
    on the 3-D mesh: ten insertion batches adding 25 % of |V| edges, then
    d_H^(0) -> d_H^(10), kappa(G0, H0), kappa(G10, H0) (H left alone),
    kappa(G10, H10) (dyGRASS updates), and the PCG iterations to a relative
    residual of 1e-8 with each sparsifier as preconditioner; beside them the
    GRASS-like H(0) of the same density (its build time, kappa and PCG
    iterations).  The CG
    iteration without preconditioner is timed for the roofline of the
    Laplacian-product path."""
    import torch
    from paper_2505_02741_b300 import dygrass as D
    from paper_2505_02741_b300 import workloads as W
    dims = tuple(int(x) for x in args.quality_mesh.split("x"))
    wl, st = W.make_mesh3d(*dims, seed=11)
    n = wl.n
    per = max(1, int(0.25 * n) // 10)
    ctx = D.Context(K=wl.K, T=wl.T, s=wl.s)
    clk = ClockSampler(0).start()
    g = ctx.load_graph(n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    h0 = g.sparsifier()
    rng = np.random.default_rng(5)
    b = rng.standard_normal(n)
    b -= b.mean()  # the mesh is connected
    db = torch.from_numpy(b).cuda()
    dx = torch.empty_like(db)
    kopt = dict(max_iter=args.lanczos_iters, check_every=10, tol=1e-6, inner_tol=1e-10,
                inner_max_iter=args.inner_max_iters)
    popt = dict(tol=1e-8, max_iter=5000, precond="sparsifier", inner_tol=1e-10, inner_max_iter=args.inner_max_iters)
    if args.quality_parts == "kappa0":  # one kappa estimate alone (a short run to profile)
        k = g.condition_number(**dict(kopt, check_every=1))
        print(json.dumps({"workload": "quality", "part": "kappa0", "n": n, "lanczos": k}), flush=True)
        ctx.close()
        return

    def measure(gr):
        k = gr.condition_number(**kopt)
        info, _ = gr.pcg_solve(db.data_ptr(), dx.data_ptr(), **popt)
        return k, info

    # the GRASS-like H(0) (reading R20) at the same density: the same spanning
    # forest plus as many off-tree edges, those of largest stretch
    tree = W.spanning_forest(n, wl.a, wl.b, wl.w)
    n_off = int(wl.h_ids.size - tree.size)
    with clk:
        d0 = g.density()
        k00, p00 = measure(g)
        gg = ctx.load_graph(n, wl.a, wl.b, wl.w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gg.init_sparsifier_grass(wl.a[tree], wl.b[tree], n_off)
        grass_ms = 1e3 * (time.perf_counter() - t0)
        kg, pg = measure(gg)
        grass = {"init_ms": grass_ms, "init_timing": "host wall clock around dg_init_sparsifier_grass (synchronous)",
                 "off_tree_edges": n_off, "d_H": gg.density()[0], "kappa": kg["kappa"], "pcg_iters": pg["iters"],
                 "lanczos": kg, "pcg": pg,
                 "compare": "H0 = the same forest + a seeded sample of as many off-tree edges: kappa_G0_H0, "
                            "pcg_iters G0_H0"}
        gg.unload()
        dens = [d0[0]]
        upd_ms = []
        for _ in range(10):
            bt = st.next_batch(per, 0)
            t0 = time.perf_counter()
            g.apply(D.make_updates(bt.u, bt.v, bt.w, bt.op))
            upd_ms.append(1e3 * (time.perf_counter() - t0))
            dens.append(g.density()[0])
        k11, p11 = measure(g)
        ga, gb, gw = g.edges()
        g2 = ctx.load_graph(n, ga, gb, gw)
        g2.init_sparsifier(h0[0], h0[1])
        k10, p10 = measure(g2)
        # plain CG: one iteration's Laplacian product and vector updates
        info_cg, _ = g.pcg_solve(db.data_ptr(), dx.data_ptr(), tol=1e-30, max_iter=args.cg_iters, precond="none")
    clk.stop()
    nnz = 2 * ga.size
    it_ms = info_cg["ms"] / max(1, info_cg["iters"])
    # algorithmic bytes of one CG iteration: the product (column id 4 B and
    # weight 8 B per stored entry; row pointer, diagonal, x_i and y_i per row)
    # and the vector passes (p.q: 2, x/r update: 5 reads+writes, r.r inside,
    # r.z with z = r: 2, p update: 3, the copy z = r: 2 -> 14 vectors of 8 B)
    alg = 12 * nnz + 28 * n + 14 * 8 * n
    peak, peak_kind = measured_peaks()
    line = {"metric": "sparsifier quality: kappa(L_G, L_H), d_H and PCG iterations (Section IV)", "workload": "quality",
            "value": p11["iters"], "unit": "PCG iterations to 1e-8 with the updated sparsifier",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"graph": f"mesh3d_{args.quality_mesh}", "n": n, "m0": wl.m, "insert_batches": 10,
                       "per_batch": per, "K": wl.K, "T": wl.T, "s": wl.s},
            "d_H": dens, "kappa": {"G0_H0": k00["kappa"], "G10_H0": k10["kappa"], "G10_H10": k11["kappa"]},
            "lanczos": {"G0_H0": k00, "G10_H0": k10, "G10_H10": k11},
            "pcg_iters": {"G0_H0": p00["iters"], "G10_H0": p10["iters"], "G10_H10": p11["iters"]},
            "pcg": {"G0_H0": p00, "G10_H0": p10, "G10_H10": p11},
            "update_ms_per_batch": upd_ms,
            "grass_init": grass,
            "cg_iteration": {"ms": it_ms, "iters": info_cg["iters"], "algorithmic_bytes": alg,
                             "roofline": {"bound": "hbm", "achieved": alg / (it_ms * 1e-3) / 1e9, "peak": peak,
                                          "unit": "GB/s", "frac": alg / (it_ms * 1e-3) / 1e9 / peak,
                                          "peak_source": peak_kind}},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--per-update-steps", type=int, default=2)
    ap.add_argument("--seq-batches", type=int, default=1,
                    help="stream batches run in the sequential (one update at a time) semantics")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work per CPU baseline")
    ap.add_argument("--ref-sample", type=int, default=500, help="reference arm: updates per step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-full-walks", action="store_true", help="skip the unpruned-walk context line (mesh)")
    ap.add_argument("--walk-shape", default="", help="fixed walk launch shape 'block,ilp' (skips the autotuner)")
    ap.add_argument("--workload", default="rmat", choices=["rmat", "mesh", "fea", "serve", "quality"],
                    help="rmat (default line), mesh, fea, serve (several graphs resident, Poisson arrivals) "
                         "or quality (kappa, d_H and PCG iterations, Section IV)")
    ap.add_argument("--quality-mesh", default="100x100x100", help="quality: mesh dimensions")
    ap.add_argument("--lanczos-iters", type=int, default=400, help="quality: Lanczos steps at most")
    ap.add_argument("--cg-iters", type=int, default=200, help="quality: timed plain CG iterations")
    ap.add_argument("--inner-max-iters", type=int, default=2000, help="quality: iterations of one L_H solve at most")
    ap.add_argument("--quality-parts", default="all", choices=["all", "kappa0"],
                    help="quality: the whole experiment, or one kappa estimate of G(0), H(0) (to profile)")
    ap.add_argument("--rmat-scale", type=int, default=22, help="rmat: log2 of the vertex count")
    ap.add_argument("--rmat-edges", type=int, default=64_000_000, help="rmat: distinct undirected edges")
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests per load point")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests of the serving summary in the default line (0: skip it)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload in ("serve", "quality"):
            args.workload = "mesh"
        return run_reference(args)
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "quality":
        return run_quality(args)

    import torch
    from paper_2505_02741_b300 import dygrass as D

    rank, world, local = dist_env()
    backend = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dev = local

    # workload (each rank an independent replica: weak scaling, no data-path collective)
    wl, st = make_workload(args.workload, args, rank)
    n_ins, n_del = BATCH[args.workload]
    L = STREAM_BATCHES[args.workload]  # the configuration's stream: L batches from G(0)
    if args.warmup > L:
        raise SystemExit(f"at most {L} warm-up steps (the stream's length)")
    batches = [st.next_batch(n_ins, n_del) for _ in range(L + args.per_update_steps)]

    ctx = D.Context(device=dev, K=wl.K, T=wl.T, s=wl.s)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    max_batch = max(len(b.u) for b in batches)
    shape = None
    coop = (1, 0)
    if args.walk_shape:
        blk, ilp = (int(x) for x in args.walk_shape.split(","))
        shape = (blk, ilp, 0, 0)

    def fresh_copy():
        """G(0) and H(0) on the device, workspace sized and steps captured up
        front; the walk shape of the warm-up copy (or the fixed one)."""
        gg = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        gg.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        if shape is not None:
            gg.set_walk_shape(shape[0], shape[1], shape[2], shape[3])
            gg.set_walk_coop(*coop)
        gg.prepare(max_batch)
        torch.cuda.synchronize()
        return gg

    def to_dev(bt):
        ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
        return ups, torch.from_numpy(ups.view(np.uint8)).to(dev)

    dev_batches = [to_dev(bt) for bt in batches]
    d_res = torch.empty(max_batch * 32, dtype=torch.uint8, device=dev)

    # warm-up: the stream's first W batches on a copy of its own (autotunes the walk)
    clk = ClockSampler(dev).start()
    g = fresh_copy()
    for k in range(args.warmup):
        ups, d_ups = dev_batches[k]
        g.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    if shape is None:
        s0 = g.stats()
        shape = (s0["walk_block"], s0["walk_ilp"], s0["walk_blocks_per_sm"], s0["walk_refill"])
        coop = (s0["walk_lanes"], s0["walk_tile"])
    tune_log = g.tune_log()
    g.unload()

    # ---- timed: device-resident batches -------------------------------------
    # step k applies stream batch k mod L; every pass of the stream starts on a
    # fresh copy at G(0) (loaded outside the timed steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    walk_ms, steps_done, valid, launches, phases = [], 0, 0, 0, []
    g = None
    for k in range(args.steps):
        if k % L == 0:
            if g is not None:
                torch.cuda.synchronize()
                clk.end()
                g.unload()
            g = fresh_copy()
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize()
            clk.begin()
        flush.fill_(float(k))  # L2 flush, outside the events
        ups, d_ups = dev_batches[k % L]
        ev[k][0].record(stream)
        g.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
        ev[k][1].record(stream)
        s = g.stats()
        walk_ms.append(s["walk_ms"])
        phases.append(s)
        steps_done += s["steps"]
        valid += s["valid"]
        launches += s["launches"]
    torch.cuda.synchronize()
    clk.end()
    clk.stop()
    if world > 1:
        dist.barrier()
    bi = args.steps % L or L  # the next stream batch for the main copy
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    (sum_valid, sum_steps), (t_max, walk_max) = reduce_over_ranks([valid, steps_done], [t_total, sum(walk_ms) / 1e3],
                                                                   world, backend)
    value = sum_valid / t_max
    walk_steps_per_s = sum_steps / walk_max

    # ---- e2e: pinned host buffers through dg_apply_updates -------------------
    # One pass of the stream on a fresh copy at G(0), through host buffers: the
    # same batches as the device-resident steps.  The step's records wait in
    # pinned host memory; the timed call copies them to the device and the
    # results back (dg_apply_updates copies pinned arrays directly).
    ge = fresh_copy()
    h_ups = torch.empty(max_batch * 24, dtype=torch.uint8, pin_memory=True).numpy().view(D.UPDATE_DTYPE)
    h_res = torch.empty(max_batch * 32, dtype=torch.uint8, pin_memory=True).numpy().view(D.RESULT_DTYPE)
    e2e_steps = min(args.steps, L)
    e2e_t, e2e_valid, e2e_nu = [], 0, 0
    for k in range(e2e_steps):
        flush.fill_(float(k))
        ups, _ = dev_batches[k]
        h_ups[: len(ups)] = ups
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ge.apply(h_ups[: len(ups)], stream=stream.cuda_stream, out=h_res)
        e2e_t.append(time.perf_counter() - t0)
        e2e_valid += int((res["status"] == 0).sum())
        e2e_nu += len(ups)
    ge.unload()
    (e2e_sum,), (e2e_tmax,) = reduce_over_ranks([e2e_valid], [sum(e2e_t)], world, backend)
    e2e = {"value": e2e_sum / e2e_tmax, "unit": "updates/s",
           "h2d_bytes_per_step": 24 * e2e_nu // e2e_steps + 16,
           "d2h_bytes_per_step": 32 * e2e_nu // e2e_steps + 96, "p50_ms": 1e3 * float(np.percentile(e2e_t, 50)),
           "p99_ms": 1e3 * float(np.percentile(e2e_t, 99)), "host_buffers": "pinned",
           "steps": e2e_steps, "batches": "one pass of the stream from G(0) on a fresh copy"}

    # ---- sequential semantics (Algorithm 1's order, one update at a time) ----
    # the stream's first batches on a fresh copy at G(0), through
    # dg_apply_updates_sequential (host records); wall clock per batch
    seq = None
    if args.seq_batches > 0:
        gs = fresh_copy()
        s_t, s_pre, s_nu = [], 0, 0
        for k in range(min(args.seq_batches, L)):
            ups, _ = dev_batches[k]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, pre = gs.apply_sequential(ups)
            s_t.append(time.perf_counter() - t0)
            s_pre += pre
            s_nu += len(ups)
        gs.unload()
        seq = {"updates_per_s": s_nu / sum(s_t), "batches": len(s_t), "updates": s_nu,
               "prefixes": s_pre, "mean_prefix": s_nu / max(1, s_pre), "ms_per_batch": 1e3 * float(np.mean(s_t)),
               "semantics": "every update sees all earlier ones (Algorithm 1); results equal one update per batch",
               "timing": "host wall clock around dg_apply_updates_sequential, stream batches from G(0)"}

    # ---- context (mesh): the same walk kernel without deletion pruning -------
    full = None
    if args.workload == "mesh" and not args.no_full_walks:
        ctx_f = D.Context(device=dev, K=wl.K, T=wl.T, s=wl.s, del_prune=False)
        gf = ctx_f.load_graph(wl.n, wl.a, wl.b, wl.w)
        gf.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        f_ms, f_steps = [], 0
        for k in range(6):
            flush.fill_(float(k))
            ups, d_ups = dev_batches[k]
            gf.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
            s = gf.stats()
            if k >= 3:
                f_ms.append(s["walk_ms"])
                f_steps += s["steps"]
        ctx_f.close()
        full = {"del_prune": False, "walk_steps_per_batch": f_steps / 3, "walk_ms": sum(f_ms) / 3,
                "walk_steps_per_s": f_steps / (sum(f_ms) / 1e3), "batches": "stream batches 4-6 on a fresh copy"}

    # ---- the one-launch-per-update form on a copy at the same state ----------
    pu = None
    if args.per_update_steps > 0:
        ga, gb, gw = g.edges()
        ha, hb, _ = g.sparsifier()
        nid = g.next_update_id
        ctx_pu = D.Context(device=dev, K=wl.K, T=wl.T, s=wl.s, walk_mode="per_update", cuda_graphs=False)
        gp = ctx_pu.load_graph(wl.n, ga, gb, gw)
        gp.init_sparsifier(ha, hb)
        gp.next_update_id = nid
        del ga, gb, gw, ha, hb
        pu_t, pu_valid, same = [], 0, True
        for k in range(args.per_update_steps):
            ups, d_ups = dev_batches[bi]
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gp.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            pu_t.append(e0.elapsed_time(e1))
            res_pu = d_res[: len(ups) * 32].cpu().numpy().copy()
            pu_valid += int(gp.stats()["valid"])
            # identical outputs: the batched form on the main graph, same batch
            g.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            same &= res_pu.tobytes() == d_res[: len(ups) * 32].cpu().numpy().tobytes()  # every byte
            bi += 1
        pu = {"updates_per_s": pu_valid / (sum(pu_t) / 1e3), "p50_ms": float(np.percentile(pu_t, 50)),
              "p99_ms": float(np.percentile(pu_t, 99)), "steps": args.per_update_steps,
              "identical_outputs": same}
        ctx_pu.close()

    # ---- roofline of the walk kernel ----------------------------------------
    peak, peak_kind = measured_peaks()
    avg_walk_s = sum(walk_ms) / 1e3 / args.steps
    steps_per_launch = steps_done / args.steps
    achieved = ALG_BYTES_PER_STEP * steps_per_launch / avg_walk_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": WALK_TRAFFIC.get(args.workload, (None, ""))[0],
            "traffic_source": WALK_TRAFFIC.get(args.workload, (None, "not captured for this workload"))[1],
            "kernel": "k_walk_batched", "bytes_per_step": ALG_BYTES_PER_STEP, "peak_source": peak_kind,
            "steps_per_launch": steps_per_launch,
            "algorithmic_bytes_per_launch": ALG_BYTES_PER_STEP * steps_per_launch,
            "gather": {"bytes_per_step": SECTOR_BYTES_PER_STEP, "walk_steps_per_s": steps_per_launch / avg_walk_s,
                       "peak_steps_per_s": peak * 1e9 / SECTOR_BYTES_PER_STEP,
                       "frac": steps_per_launch / avg_walk_s / (peak * 1e9 / SECTOR_BYTES_PER_STEP)}}

    # ---- roofline of the list merge (G's touched lists) ----------------------
    # every entry of a touched list is read once from the old list and written
    # once to the new one: 32 B each way; CUDA events around the merge kernel
    # inside the captured step (G's merge runs beside H's on the second stream)
    merge = None
    m_ms = [p["merge_ms"] for p in phases]
    if all(x > 0 for x in m_ms):
        m_entries = float(np.mean([p["merge_entries"] for p in phases]))
        m_s = sum(m_ms) / 1e3 / len(m_ms)
        m_ach = MERGE_BYTES_PER_ENTRY * m_entries / m_s / 1e9
        merge = {"bound": "hbm", "achieved": m_ach, "peak": peak, "unit": "GB/s", "frac": m_ach / peak,
                 "traffic": MERGE_TRAFFIC.get(args.workload, (None, ""))[0],
                 "traffic_source": MERGE_TRAFFIC.get(args.workload, (None, "not captured for this workload"))[1],
                 "kernel": "k_exec_merge (G's touched lists)", "bytes_per_entry": MERGE_BYTES_PER_ENTRY,
                 "entries_per_launch": m_entries, "ms_per_launch": 1e3 * m_s, "peak_source": peak_kind,
                 "algorithmic_bytes_per_launch": MERGE_BYTES_PER_ENTRY * m_entries}

    serving = None
    if rank == 0 and args.serve_requests > 0:
        r = serve_experiment((0.6,), args.serve_requests)
        pt = r["loads"]["0.6"]
        serving = {"offered_load": 0.6, "requests": pt["requests"], "updates_per_s": pt["updates_per_s"],
                   "latency_ms": pt["latency_ms"], "queue_ms": pt["queue_ms"],
                   "per_graph_p99_ms": {n: v["latency_ms"]["p99"] for n, v in pt["per_graph"].items()},
                   "per_update_form": r["per_update_form"],
                   "graphs": "grid 64x64, mesh 100^3, FEA 2048^2 resident together (--workload serve: 30/60/90 %)"}

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu:
        # the stream goes on past the timed batches for as long as the CPU needs
        more = (st.next_batch(n_ins, n_del) for _ in range(100_000))
        cpu, cpu_all = oracle_baseline(wl, itertools.chain(batches, more), args.cpu_budget)
        cpu.update(host_cpu())
        cpu["all_cores"] = cpu_all

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "batch": n_ins + n_del, "insertions": n_ins,
                       "deletions": n_del, "K": wl.K, "T": wl.T, "s": wl.s, "parallelism": f"replicas{world}",
                       "l2": "flushed (256 MB write) between timed steps",
                       "stream": f"{L} batches from G(0); timed step k applies batch k mod {L}, each pass on a "
                                 f"fresh copy ({-(-args.steps // L)} passes)"},
            "walk_steps_per_s": walk_steps_per_s,
            "per_batch": {"walk_steps": steps_done / args.steps,
                          "d_H_first_pass": [p["h_edges"] / wl.n - 1.0 for p in phases[:L]],
                          "walked_updates": float(np.mean([p["walked"] for p in phases])),
                          "phase_ms": {k: float(np.mean([p[k] for p in phases])) for k in
                                       ("mutate_ms", "walk_ms", "reduce_ms", "emit_ms", "commit_ms", "batch_ms")},
                          "walk_shape": {"block": phases[-1]["walk_block"], "ilp": phases[-1]["walk_ilp"],
                                         "blocks_per_sm": phases[-1]["walk_blocks_per_sm"],
                                         "refill": phases[-1]["walk_refill"], "lanes": phases[-1]["walk_lanes"],
                                         "tile": phases[-1]["walk_tile"], "autotuned": not args.walk_shape,
                                         "autotuner_trials": [dict(d, ms=round(ms, 4)) for d, ms in tune_log]},
                          "launches": launches / args.steps, "cuda_graph": bool(phases[-1]["graph_replayed"])},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "per_update_form": pu,
            "sequential": seq,
            "roofline": roof,
            "roofline_merge": merge,
            "roofline_full_walks": full,
            "cpu_baseline": cpu,
            "serving": serving,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
