"""Benchmark: batched dyGRASS updates on the 3-D power-grid-like mesh.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload: 100x100x100 mesh (1M vertices, 2.97M edges, w = 10^U(-2,2), z edges
x5), H(0) = max-weight spanning forest + 10 % of the off-tree edges, K = 100,
T = 100, s = 32.  One step = one batch of 10k insertions (<= 6 hops apart) and
10k deletions of current edges, shuffled.  Synthetic data, seeded.

value    : updates/s of the batched form, batches already resident in HBM
           (dg_apply_updates_device), CUDA events on the batch stream, L2
           flushed (256 MB write) between steps.
e2e      : the same through dg_apply_updates with host buffers (H2D of the
           batch, D2H of the results inside the timed region).
roofline : the walk kernel, algorithmic bytes = 32 B (one DRAM sector) per
           useful walk step, against the measured HBM copy bandwidth.
Also reported: walk-steps/s, the one-launch-per-update form at identical
outputs, per-batch latency p50/p99 of both forms, and the CPU oracle on a
bounded sample of the same workload.

Under torchrun each rank runs an independent replica (its own seed); there is
no collective on the data path; rank 0 prints the whole-job line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "updates/s & walk-steps/s on 1 B300, batched vs per-update; p50/p99 latency"
BYTES_PER_STEP = 32  # one 32-byte DRAM sector per walk step (the entry holds nbr, next list, rev, r)
N_INS, N_DEL = 10_000, 10_000
# DRAM bytes (read + write) of one walk launch of this workload, from one ncu
# capture of the current walk kernel (cold L2), or None while the kernel has
# changed since its last capture.
WALK_TRAFFIC_BYTES = None
WALK_TRAFFIC_SOURCE = ("stale: the walk kernel changed after its last capture (profiles/walk_k_walk_batched_mesh3d_100.md "
                       "measured 2.735e8 B per launch before the fallback queue claimed long lists)")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, local=0):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.index = ids[local] if local < len(ids) else str(local)
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


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


def oracle_sample(wl, batches, budget_s=20.0):
    """The CPU oracle as it stands, single-threaded, on the first batches of the
    same stream until about budget_s of CPU work: updates/s."""
    from oracle.oracle import OracleGraph
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    done, t_total, steps, nb = 0, 0.0, 0, 0
    for bt in batches:
        t0 = time.perf_counter()
        r = o.apply(bt.u, bt.v, bt.w, bt.op)
        t_total += time.perf_counter() - t0
        done += int((r["status"] == 0).sum())
        steps += int(r["steps"].sum())
        nb += 1
        if t_total >= budget_s:
            break
    o.close()
    return done / t_total, steps / t_total, nb, t_total


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload, bounded per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_02741_b300 import workloads as W
    from oracle.oracle import OracleGraph
    wl, st = W.make_mesh3d(seed=0)
    o = OracleGraph(wl.n, wl.a, wl.b, wl.w, K=wl.K, T=wl.T, s=wl.s)
    o.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    # each step: a bounded sample (the first 2,000 updates of a 20k batch) so the run stays short
    sample = 2000
    times, units = [], 0
    for i in range(args.warmup + args.steps):
        bt = st.next_batch(N_INS, N_DEL)
        t0 = time.perf_counter()
        r = o.apply(bt.u[:sample], bt.v[:sample], bt.w[:sample], bt.op[:sample])
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            units += int((r["status"] == 0).sum())
    value = units / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "batch": sample,
                                            "K": wl.K, "T": wl.T, "s": wl.s},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {sample} updates of each 20k-update batch, single thread"},
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


def run_serve(args):
    """Serving: the 64x64 grid, the 100^3 mesh and the 2048^2 FEA-like mesh
    resident at once.  Per graph a Poisson request stream, batch sizes
    floor(exp(U(0, ln 50001))) (clipped for the small grid), 50/50
    insertions/deletions.  The three streams share the GPU, so each is offered
    at `load` x its graph's capacity measured alone, divided by the number of
    graphs.  Reports updates/s and p50/p99 request latency (submit to results
    on the host) beside the one-launch-per-update form on a sample of requests."""
    import torch
    from paper_2505_02741_b300 import dygrass as D
    from paper_2505_02741_b300 import workloads as W

    torch.cuda.init()
    specs = [("grid64", lambda: W.make_grid(64, 64, seed=0), 400),
             ("mesh100", lambda: W.make_mesh3d(seed=0), 50_000),
             ("fea2048", lambda: W.make_fea(seed=0), 50_000)]
    arr_rng = W.rngs(7)["arrivals"]
    per_graph = max(4, args.requests // len(specs))
    graphs = []
    for name, mk, cap in specs:
        wl, st = mk()
        _, sizes = W.serving_arrivals(per_graph, 1.0, arr_rng)
        sizes = np.minimum(sizes, cap)
        if name == "grid64":
            reqs = []
            for s in sizes:
                ins = int(s) // 2
                b = st.next_batch(ins, int(s) - ins)
                reqs.append((b.u, b.v, b.w, b.op))
        else:
            total = int(sizes.sum())
            big = st.next_batch(total // 2, total - total // 2)
            reqs = _split_requests(big, sizes)
        graphs.append((name, wl, reqs))

    def load(ctx, wl):
        g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
        g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
        return g

    # batched capacity per graph, on its own copy (first requests, sequential)
    cap_ups = {}
    for name, wl, reqs in graphs:
        ctx = D.Context()
        g = load(ctx, wl)
        done, t_tot = 0, 0.0
        for r in reqs[:3]:  # warm-up: workspace, captured steps, autotuner
            g.apply(D.make_updates(*r))
        for r in reqs[3: min(15, len(reqs))]:
            ups = D.make_updates(*r)
            t0 = time.perf_counter()
            g.apply(ups)
            dt = time.perf_counter() - t0
            done += len(ups)
            t_tot += dt
        cap_ups[name] = done / t_tot
        ctx.close()

    # the served stream
    ctx = D.Context()
    gs = {name: load(ctx, wl) for name, wl, _ in graphs}
    schedule = []
    for name, _, reqs in graphs:
        mean = float(np.mean([len(r[0]) for r in reqs]))
        lam = args.load * cap_ups[name] / len(graphs) / mean  # requests / s (the GPU is shared)
        t = np.cumsum(arr_rng.exponential(1.0 / lam, size=len(reqs)))
        for k, r in enumerate(reqs):
            schedule.append((float(t[k]), name, k, D.make_updates(*r)))
    schedule.sort(key=lambda x: x[0])
    tickets = []
    t_start = time.perf_counter()
    for at, name, k, ups in schedule:
        delay = at - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        tickets.append((name, k, len(ups)) + gs[name].submit(ups))
    lat, units = [], 0
    for name, k, nu, ticket, _res in tickets:
        res, ms = gs[name].wait(ticket, timeout_ms=600000)
        lat.append(ms)
        units += int((res["status"] == 0).sum())
    wall = time.perf_counter() - t_start
    ctx.close()

    # the one-launch-per-update form on a sample of the mesh requests
    name, wl, reqs = graphs[1]
    ctx = D.Context(walk_mode="per_update", cuda_graphs=False)
    g = load(ctx, wl)
    pu_lat, pu_units = [], 0
    for r in reqs[:6]:
        ups = D.make_updates(*r)
        t0 = time.perf_counter()
        res = g.apply(ups)
        pu_lat.append(1e3 * (time.perf_counter() - t0))
        pu_units += int((res["status"] == 0).sum())
    ctx.close()

    line = {"metric": "serving: updates/s and p50/p99 request latency", "workload": "serve",
            "value": units / wall, "unit": "updates/s", "n_gpus": 1, "requests": len(tickets),
            "offered_load": args.load, "offered_per_graph": "load x capacity alone / 3 (one GPU shared)",
            "capacity_updates_per_s": cap_ups,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(np.max(lat))},
            "graphs": {n: {"n": wl.n, "m": wl.m, "requests": len(r)} for n, wl, r in graphs},
            "per_update_form": {"graph": "mesh100", "requests": len(pu_lat),
                                "updates_per_s": pu_units / (sum(pu_lat) / 1e3),
                                "p50_ms": float(np.percentile(pu_lat, 50)), "p99_ms": float(np.percentile(pu_lat, 99))},
            "dtype": "f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--per-update-steps", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-full-walks", action="store_true", help="skip the unpruned-walk context line")
    ap.add_argument("--walk-shape", default="", help="fixed walk launch shape 'block,ilp' (skips the autotuner)")
    ap.add_argument("--workload", default="mesh", choices=["mesh", "fea", "rmat", "serve"],
                    help="mesh (default line), fea, rmat, or serve (several graphs resident, Poisson arrivals)")
    ap.add_argument("--rmat-scale", type=int, default=22, help="rmat: log2 of the vertex count")
    ap.add_argument("--rmat-edges", type=int, default=64_000_000, help="rmat: distinct undirected edges")
    ap.add_argument("--load", type=float, default=0.6, help="serve: offered load as a fraction of capacity")
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests in the measured stream")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.workload == "serve":
        return run_serve(args)

    import torch
    from paper_2505_02741_b300 import dygrass as D
    from paper_2505_02741_b300 import workloads as W

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
    n_ins, n_del = N_INS, N_DEL
    if args.workload == "fea":  # one batch of 100k mixed updates per step
        wl, st = W.make_fea(seed=rank)
        n_ins, n_del = 50_000, 50_000
    elif args.workload == "rmat":  # 50k updates per step, 60 % insertions
        wl, st = W.make_rmat(scale=args.rmat_scale, n_edges=args.rmat_edges, seed=rank)
        n_ins, n_del = 30_000, 20_000
    else:
        wl, st = W.make_mesh3d(seed=rank)
    n_batches = args.warmup + args.steps + args.steps + args.per_update_steps
    batches = [st.next_batch(n_ins, n_del) for _ in range(n_batches)]

    ctx = D.Context(device=dev, K=wl.K, T=wl.T, s=wl.s)
    g = ctx.load_graph(wl.n, wl.a, wl.b, wl.w)
    g.init_sparsifier(wl.a[wl.h_ids], wl.b[wl.h_ids])
    if args.walk_shape:
        blk, ilp = (int(x) for x in args.walk_shape.split(","))
        g.set_walk_shape(blk, ilp, 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def to_dev(bt):
        ups = D.make_updates(bt.u, bt.v, bt.w, bt.op)
        return ups, torch.from_numpy(ups.view(np.uint8)).to(dev)

    dev_batches = [to_dev(bt) for bt in batches]
    d_res = torch.empty(max(len(b) for b in batches) * 32, dtype=torch.uint8, device=dev)

    bi = 0
    for _ in range(args.warmup):
        ups, d_ups = dev_batches[bi]
        g.apply_device(d_ups.data_ptr(), len(ups), d_res.data_ptr(), stream.cuda_stream)
        bi += 1
    torch.cuda.synchronize()

    # ---- timed: device-resident batches -------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    walk_ms, steps_done, valid, launches, phases = [], 0, 0, 0, []
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))  # L2 flush, outside the events
            ups, d_ups = dev_batches[bi]
            bi += 1
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
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    (sum_valid, sum_steps), (t_max, walk_max) = reduce_over_ranks([valid, steps_done], [t_total, sum(walk_ms) / 1e3],
                                                                   world, backend)
    value = sum_valid / t_max
    walk_steps_per_s = sum_steps / walk_max

    # ---- e2e: host buffers through dg_apply_updates --------------------------
    # the step's records wait in pinned host memory; the timed call copies them to
    # the device and the results back (dg_apply_updates copies pinned arrays directly)
    nmax = max(len(b) for b in batches)
    h_ups = torch.empty(nmax * 24, dtype=torch.uint8, pin_memory=True).numpy().view(D.UPDATE_DTYPE)
    h_res = torch.empty(nmax * 32, dtype=torch.uint8, pin_memory=True).numpy().view(D.RESULT_DTYPE)
    e2e_t, e2e_valid, e2e_nu = [], 0, 0
    for k in range(args.steps):
        flush.fill_(float(k))
        ups, _ = dev_batches[bi]
        bi += 1
        h_ups[: len(ups)] = ups
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = g.apply(h_ups[: len(ups)], stream=stream.cuda_stream, out=h_res)
        e2e_t.append(time.perf_counter() - t0)
        e2e_valid += int((res["status"] == 0).sum())
        e2e_nu += len(ups)
    (e2e_sum,), (e2e_tmax,) = reduce_over_ranks([e2e_valid], [sum(e2e_t)], world, backend)
    e2e = {"value": e2e_sum / e2e_tmax, "unit": "updates/s",
           "h2d_bytes_per_step": 24 * e2e_nu // args.steps + 16,
           "d2h_bytes_per_step": 32 * e2e_nu // args.steps + 96, "p50_ms": 1e3 * float(np.percentile(e2e_t, 50)),
           "p99_ms": 1e3 * float(np.percentile(e2e_t, 99)), "host_buffers": "pinned"}

    # ---- context: the same walk kernel without deletion pruning ---------------
    # (every deletion walker runs to its own stop, as Algorithm 1 walks them):
    # a fresh copy of the graph takes the stream's first batches; the walk is
    # then bandwidth-bound rather than bound by the chain of the longest walks
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
        f_bytes = BYTES_PER_STEP * f_steps / 3
        f_ach = f_bytes / (sum(f_ms) / 3 / 1e3) / 1e9
        full = {"del_prune": False, "walk_steps_per_batch": f_steps / 3, "walk_ms": sum(f_ms) / 3,
                "walk_steps_per_s": f_steps / (sum(f_ms) / 1e3), "achieved_gbs": f_ach,
                "frac": f_ach / measured_peaks()[0], "batches": "stream batches 4-6 on a fresh copy"}

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
            # every field but steps (pruned deletion walkers stop at scheduling-dependent steps)
            r0 = res_pu.view(D.RESULT_DTYPE)
            r1 = d_res[: len(ups) * 32].cpu().numpy().view(D.RESULT_DTYPE)
            same &= all(np.array_equal(np.ascontiguousarray(r0[f]).view(np.uint8),
                                       np.ascontiguousarray(r1[f]).view(np.uint8))
                        for f in D.RESULT_DTYPE.names if f != "steps")
            bi += 1
        pu = {"updates_per_s": pu_valid / (sum(pu_t) / 1e3), "p50_ms": float(np.percentile(pu_t, 50)),
              "p99_ms": float(np.percentile(pu_t, 99)), "steps": args.per_update_steps,
              "identical_outputs": same}
        ctx_pu.close()

    # ---- roofline of the walk kernel ----------------------------------------
    peak, peak_kind = measured_peaks()
    avg_walk_s = sum(walk_ms) / 1e3 / args.steps
    bytes_per_launch = BYTES_PER_STEP * steps_done / args.steps
    achieved = bytes_per_launch / avg_walk_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": WALK_TRAFFIC_BYTES if args.workload == "mesh" else None,
            "traffic_source": WALK_TRAFFIC_SOURCE if args.workload == "mesh" else None, "kernel": "k_walk_batched",
            "bytes_per_step": BYTES_PER_STEP, "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": bytes_per_launch}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu_v, cpu_steps, nb, tt = oracle_sample(wl, batches[: 2], args.cpu_budget)
        cpu = {"value": cpu_v, "unit": "updates/s", "cores": 1, "kind": "oracle",
               "sample": f"{nb} full batch(es) of 20k updates from the start of the stream, {tt:.1f} s",
               "walk_steps_per_s": cpu_steps}

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "batch": n_ins + n_del, "insertions": n_ins,
                       "deletions": n_del, "K": wl.K, "T": wl.T, "s": wl.s, "parallelism": f"replicas{world}",
                       "l2": "flushed (256 MB write) between timed steps"},
            "walk_steps_per_s": walk_steps_per_s,
            "per_batch": {"walk_steps": steps_done / args.steps,
                          "walked_updates": float(np.mean([p["walked"] for p in phases])),
                          "phase_ms": {k: float(np.mean([p[k] for p in phases])) for k in
                                       ("mutate_ms", "walk_ms", "reduce_ms", "emit_ms", "commit_ms", "batch_ms")},
                          "walk_shape": {"block": phases[-1]["walk_block"], "ilp": phases[-1]["walk_ilp"],
                                         "blocks_per_sm": phases[-1]["walk_blocks_per_sm"],
                                         "cut": phases[-1]["walk_cut"], "autotuned": True},
                          "launches": launches / args.steps, "cuda_graph": bool(phases[-1]["graph_replayed"])},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "per_update_form": pu,
            "roofline": roof,
            "roofline_full_walks": full,
            "cpu_baseline": cpu,
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
