"""Benchmark of the WBPR max-flow hot path on GB300.

Workload (one GPU): R-MAT scale 20, edge factor 16 (a,b,c,d = .57,.19,.19,.05),
self-loops and duplicates removed (16.09 M arcs), capacities U[1,1000],
s = largest out-degree, t = largest in-degree; seeded, synthetic (stands in
for the power-law SNAP graphs of the paper's Table 1).

One step = the whole hot path on that input, graph arrays resident in HBM:
  build the BCSR residual graph (with reverse index) from device COO arrays,
  maximum flow (preflow, push-relabel iterations with global relabel and gap,
  phase 2 returning excess to s, per-arc flows), minimum cut (source side and
  capacity), release.
value = residual arcs scanned per second over the timed steps (entries read
by the min-height scans of Alg. 2, both phases; see wbpr_stats).

--impl reference times the CPU oracle (FIFO push-relabel) on a bounded sample
of the same workload (R-MAT scale 18, same parameters) on the host.
Under torchrun (N > 1) every rank solves its own replica (a single max-flow
instance does not shard); value = the arcs all ranks scanned / the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual arcs scanned/s (R-MAT 20 max-flow + min-cut, BCSR)"
UNIT = "arcs/s"

# The library's own kernels per step: the BCSR build (half_keys, tail_caps,
# scatter_prefix, run_heads, merge_runs, pair_slots, max_degree_kernel),
# solve_kernel for the flow and for the cut, and edge_flow_kernel.  CUB's
# sort and scan kernels come on top.
LAUNCHES_PER_STEP = 10

# Algorithmic bytes per unit of the BCSR solver (each unit is counted by the
# kernel itself, see wbpr_get_stats).
B_ENTRY = 12          # BCSR entry scanned: col 4 + cf 4 + h[col] 4
B_ACTIVE = 36         # per AVQ entry: offsets 16, e 8, h 4, queue write 4 + read 4
B_AVQ_SCAN = 12       # per vertex per iteration: e 8 + h 4
B_PUSH = 52           # cf[k], cf[rev], cfb[k], cfb[rev] int32 RMW (32) + e(v) int64 RMW (16) + rev 4
B_RELABEL = 4
B_GR_ENTRY = 12       # col 4 + cfb 4 (mirrored reverse residual) + h 4
B_GR_VERTEX = 12      # per vertex per global relabel: h init/finalize, dead, queue


def algorithmic_bytes(st: dict, n: int) -> int:
    return (B_ENTRY * st["arcs_scanned"] + B_ACTIVE * st["active_total"] +
            B_AVQ_SCAN * n * st["iterations"] + B_PUSH * st["pushes"] +
            B_RELABEL * st["relabels"] + B_GR_ENTRY * st["gr_arcs_scanned"] +
            B_GR_VERTEX * n * st["global_relabels"])


def profiled_traffic():
    """DRAM bytes (read + write) of one solve launch from the committed ncu
    summary, or None when the solver's device code (solver_impl.cuh) changed
    since that capture."""
    import hashlib
    import re
    try:
        with open(os.path.join(ROOT, "profiles", "solve_kernel_rmat20.md")) as f:
            text = f.read()
        with open(os.path.join(ROOT, "paper_2404_00270_gb300", "csrc", "solver_impl.cuh"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        tag = re.search(r"sha256 prefix `([0-9a-f]+)`", text).group(1)
        if not sha.startswith(tag):
            return None
        rd = int(re.search(r"dram__bytes_read\.sum \| ([\d,]+) B", text).group(1).replace(",", ""))
        wr = int(re.search(r"dram__bytes_write\.sum \| ([\d,]+) B", text).group(1).replace(",", ""))
        return rd + wr
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, flag in zip(names, p[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms: float, units: float, device=None):
    """Whole-job figures over all ranks: the slowest rank's time and the sum
    of the units every rank processed (replicas only: no data exchange)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(uu)
    return float(tt.item()), float(uu.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_sample(seconds_budget: float = 20.0, scale: int = 18):
    """The oracle, as it stands, on a bounded sample: R-MAT `scale`."""
    import oracle
    import workloads as W
    oracle.build()
    g = W.rmat(scale, 16, 2)
    src, dst, cap = g.numpy()
    runs, arcs, secs = 0, 0, 0.0
    while secs < seconds_budget or runs == 0:
        t0 = time.perf_counter()
        r = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=True, want_cut=True)
        secs += time.perf_counter() - t0
        arcs += r["stats"]["arcs_scanned"]
        runs += 1
        if runs >= 3 and secs > seconds_budget / 2:
            break
    return {"value": arcs / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale {scale} (edge factor 16, seed 2, {g.m} arcs), FIFO push-relabel "
                      f"phase 1 + 2 + cut, {runs} solves in {secs:.1f} s, 1 thread",
            "time_to_solution_s": secs / runs}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    g = W.rmat(18, 16, 2)
    src, dst, cap = g.numpy()
    times, arcs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=True, want_cut=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            arcs.append(r["stats"]["arcs_scanned"])
    total = sum(times)
    value = sum(arcs) / total
    sample = f"R-MAT scale 18 (edge factor 16, seed 2, {g.m} arcs) per step, oracle phase 1 + 2 + cut"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "rmat18-sample-of-rmat20", "layout": "adjacency list (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_2404_00270_gb300 as wb
    import workloads as W
    wb.load()
    wb.use_torch_allocator(True)
    stream = torch.cuda.current_stream()

    g = W.rmat(args.scale, 16, 2, device=dev)
    n, m, s, t = g.n, g.m, g.s, g.t
    flow = torch.empty(m, dtype=torch.int32, device=dev)
    side = torch.empty(n, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step(layout):
        G = wb.wbpr_build(n, m, g.src, g.dst, g.cap, s, t, layout, None, stream)
        v = wb.wbpr_maxflow(G, stream, flow)
        st = wb.wbpr_get_stats(G)
        c = wb.wbpr_mincut(G, stream, side)
        G.close()
        return v, c, st

    # warm-up
    for _ in range(args.warmup):
        v0, c0, _ = step(wb.WBPR_BCSR)
    assert v0 == c0

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    arcs = 0
    solve_ms = 0.0
    alg_bytes = 0
    value_seen = None
    for _ in range(args.steps):
        v, c, st = step(wb.WBPR_BCSR)
        arcs += st["arcs_scanned"]
        solve_ms += st["solve_ms"]
        alg_bytes += algorithmic_bytes(st, n)
        value_seen = v
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms, arcs_all = aggregate_ranks(ms, float(arcs), dev)
    value = arcs_all / (ms / 1e3)

    # time-to-maxflow with the graph resident (phase 1, value only), both layouts
    breakdown = {}
    for name, layout in (() if args.quick else (("bcsr", wb.WBPR_BCSR), ("rcsr", wb.WBPR_RCSR))):
        torch.cuda.synchronize()
        tb = time.perf_counter()
        G = wb.wbpr_build(n, m, g.src, g.dst, g.cap, s, t, layout, None, stream)
        torch.cuda.synchronize()
        build_ms = 1e3 * (time.perf_counter() - tb)
        reps = 3
        vals, t_ms, arcs_l = [], [], []
        for _ in range(reps):
            vals.append(wb.wbpr_maxflow(G, stream))
            st = wb.wbpr_get_stats(G)
            t_ms.append(st["solve_ms"])
            arcs_l.append(st["arcs_scanned"])
        wb.wbpr_maxflow(G, stream, flow)
        st2 = wb.wbpr_get_stats(G)
        info = wb.wbpr_get_info(G)
        G.close()
        breakdown[name] = {"value": vals[0], "time_to_maxflow_ms": statistics.median(t_ms),
                           "arcs_per_s": statistics.median(arcs_l) / (statistics.median(t_ms) / 1e3),
                           "build_ms": build_ms, "phase1_plus_phase2_ms": st2["solve_ms"],
                           "iterations": st2["iterations"], "global_relabels": st2["global_relabels"],
                           "device_bytes": info["device_bytes"], "grid_blocks": info["grid_blocks"]}
        assert len(set(vals)) == 1 and vals[0] == value_seen

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hsrc = g.src.cpu().pin_memory()
    hdst = g.dst.cpu().pin_memory()
    hcap = g.cap.cpu().pin_memory()
    hflow = torch.empty(m, dtype=torch.int32).pin_memory()
    hside = torch.empty(n, dtype=torch.uint8).pin_memory()
    e_steps = 0 if args.quick else max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    e_arcs = 0
    for _ in range(e_steps):
        G = wb.wbpr_build(n, m, hsrc, hdst, hcap, s, t, wb.WBPR_BCSR, None, stream)
        v = wb.wbpr_maxflow(G, stream, hflow)
        e_arcs += wb.wbpr_get_stats(G)["arcs_scanned"]
        c = wb.wbpr_mincut(G, stream, hside)
        G.close()
    barrier()
    e_ms = 1e3 * (time.perf_counter() - t0)
    e2e = {"value": e_arcs / (e_ms / 1e3) * (world if world > 1 else 1) if e_steps else None,
           "unit": UNIT, "h2d_bytes_per_step": 12 * m, "d2h_bytes_per_step": 4 * m + n + 16,
           "ms_per_step": e_ms / e_steps if e_steps else None}

    peak, peak_kind = measured_peaks()
    launch_ms = solve_ms / args.steps
    achieved = (alg_bytes / args.steps) / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic() if args.scale == 20 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}-maxflow-mincut", "scale": args.scale, "edge_factor": 16,
                   "n": n, "m": m, "s": s, "t": t, "layout": "bcsr+rev",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": (f"inputs larger than L2 (COO {12 * m / 1e6:.0f} MB"
                          + (f", BCSR handle {breakdown['bcsr']['device_bytes'] / 1e6:.0f} MB" if breakdown else "")
                          + " per step)"),
                   "flow_value": value_seen,
                   "time_to_maxflow_ms": breakdown["bcsr"]["time_to_maxflow_ms"] if breakdown else None,
                   "layouts": breakdown},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "solve_kernel",
                     "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})"},
        "gpu_launches": args.steps * LAUNCHES_PER_STEP,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """The batched / served workload: a seeded mix of grids and bipartite
    graphs of uneven size, solved (a) one instance per launch, (b) all in one
    batched launch, (c) through the continuous-batching server with Poisson
    arrivals."""
    import numpy as np
    import torch
    import paper_2404_00270_gb300 as wb
    from paper_2404_00270_gb300 import serve
    import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wb.load()
    wb.use_torch_allocator(True)
    stream = torch.cuda.current_stream()
    specs = W.batch_spec(args.batch_count)
    t0 = time.perf_counter()
    insts = [W.make_from_spec(sp, device=dev) for sp in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    total_arcs = sum(g.m for g in insts)
    t0 = time.perf_counter()
    graphs = [wb.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, wb.WBPR_BCSR, None, stream) for g in insts]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # (a) one instance per launch, on an evenly spaced sample
    step = max(1, len(graphs) // args.plain_sample)
    sample = list(range(0, len(graphs), step))
    plain_ms, plain_vals = [], {}
    for i in sample:
        torch.cuda.synchronize()
        ta = time.perf_counter()
        plain_vals[i] = wb.wbpr_maxflow(graphs[i], stream)
        plain_ms.append(1e3 * (time.perf_counter() - ta))
    plain_rate = len(sample) / (sum(plain_ms) / 1e3)
    # (b) the whole mix in one batched launch per step
    for _ in range(args.warmup):
        vals = wb.wbpr_maxflow_batch(graphs, stream)
    assert all(vals[i] == plain_vals[i] for i in sample)
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        vals = wb.wbpr_maxflow_batch(graphs, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    batch_rate = len(graphs) / (ms / 1e3)
    inst_ms = [wb.wbpr_get_stats(G)["solve_ms"] for G in graphs]
    slowest = sorted(range(len(graphs)), key=lambda i: -inst_ms[i])[:5]
    slowest = [{"spec": list(specs[i]), "ms": inst_ms[i], "team_blocks": wb.wbpr_get_info(graphs[i])["grid_blocks"]}
               for i in slowest]
    for G in graphs:
        G.close()
    del graphs
    torch.cuda.empty_cache()
    # (c) continuous batching with Poisson arrivals at a fraction of the batch rate
    serving = {}
    rng = np.random.default_rng(5)
    n_serve = min(len(insts), args.serve_count)
    for frac in args.serve_rates:
        lam = frac * batch_rate
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_serve))
        reqs = [serve.Request(i, g.n, g.src, g.dst, g.cap, g.s, g.t, float(a))
                for i, (g, a) in enumerate(zip(insts[:n_serve], arrivals))]
        free_b, _ = torch.cuda.mem_get_info()
        srv = serve.Server(int(0.5 * free_b))
        out = srv.run(reqs)
        bad = [r.rid for r in out if r.rid in plain_vals and r.value != plain_vals[r.rid]]
        assert not bad, bad
        summ = serve.latency_summary(out)
        summ["rate_per_s"] = lam
        serving[f"{frac:g}x"] = summ
    line = {
        "metric": f"batched solves/s ({len(insts):,}-instance mix, one batched launch)", "value": batch_rate,
        "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batch-mix-{len(insts)}", "instances": len(insts), "arcs": total_arcs,
                   "generate_s": gen_s, "build_s": build_s, "layout": "bcsr+rev",
                   "plain_solves_per_s": plain_rate, "plain_sample": len(sample),
                   "plain_p50_ms": float(np.percentile(plain_ms, 50)),
                   "plain_p99_ms": float(np.percentile(plain_ms, 99)),
                   "speedup_vs_plain": batch_rate / plain_rate,
                   "batch_ms": ms, "slowest_in_batch": slowest, "serving": serving},
        "roofline": None, "clocks": clocks,
        "gpu_launches": args.steps * 2,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wbpr", choices=["wbpr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (20 = the benchmark workload)")
    ap.add_argument("--quick", action="store_true", help="timed steps only (profiling runs)")
    ap.add_argument("--workload", default="rmat20", choices=["rmat20", "batch"])
    ap.add_argument("--batch-count", type=int, default=1024)
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--serve-count", type=int, default=512)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[0.5, 1.0])
    args = ap.parse_args()
    if args.workload == "batch" and args.impl != "reference":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
