"""Benchmark of the WBPR max-flow hot path on GB300.

Headline workload (one GPU): R-MAT scale 26, edge factor 16 (a,b,c,d = .57,
.19,.19,.05), self-loops and duplicates removed (1.06 G arcs), capacities
U[1, 10^4], s = largest out-degree, t = largest in-degree, seed 4; seeded and
synthetic (it stands in for the massive power-law SNAP graphs of the
paper's Table 1).  BCSR with the reverse index, int64 excesses.

One step = the whole hot path on that input, COO arrays resident in HBM:
  build the BCSR residual graph from the device COO arrays, maximum flow
  (preflow, push-relabel iterations with global relabel and gap, phase 2
  returning excess to s, per-arc flows), minimum cut (source side and
  capacity), release.
value = residual arcs scanned per second over the timed steps (entries read
by the min-height scans of Alg. 2, both phases; see wbpr_stats).

Beside it, in `config`: the R-MAT 20 workload in both layouts (time to
maximum flow, build, phase 1 + 2), the handle's HBM footprint against the
O(V^2) adjacency matrix, the oracle's offline value for the R-MAT 26 graph,
and a compact batch / serving block on the seeded mix of grids and
bipartite graphs.  `cpu_baseline` times the oracle on the R-MAT 20 graph on
one host core and reports both arms' time to solution on that same graph.

--impl reference times the CPU oracle (FIFO push-relabel) per step on a
bounded sample of the same workload family (R-MAT scale 18, same
parameters) on the host.  --workload rmat20 makes R-MAT 20 the headline;
--workload batch runs the batched / served mix alone.
Under torchrun (N > 1) every rank solves its own replica (a single max-flow
instance does not shard); value = the arcs all ranks scanned / the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "arcs/s"
WORKLOADS = {
    "rmat26": dict(scale=26, seed=4, cap_hi=10000),
    "rmat22": dict(scale=22, seed=2, cap_hi=1000),   # a small case of the same kernel, for profiling
    "rmat20": dict(scale=20, seed=2, cap_hi=1000),
}

# The library's own kernels per step: the BCSR build (validate_keys, in_prep,
# merge_runs4, rev_pairs4, max_degree_kernel; merge_runs and rev_pairs as
# well when the half-entry count 2m' is not a multiple of four (m' = non-loop
# arcs; the R-MAT workloads have no self-loops, so m' = m); scatter_prefix
# only for inputs with parallel arcs, which the R-MAT workloads have not;
# count_degrees_warp, iota_u32, invert_order when the handle is renumbered),
# solve_kernel for the flow and for the cut, and edge_flow_kernel.  CUB's
# sort, merge and scan kernels come on top.
def launches_per_step(renumbered: bool, m: int) -> int:
    return 8 + (2 if m % 2 else 0) + (3 if renumbered else 0)


# Algorithmic bytes per unit of the BCSR solver (each unit is counted by the
# kernel itself, see wbpr_get_stats).
B_ENTRY = 12          # BCSR entry scanned: col 4 + cf 4 + h[col] 4
B_ACTIVE = 36         # per AVQ entry: offsets 16, e 8, h 4, queue write 4 + read 4
B_AVQ_SCAN = 12       # per vertex per iteration: e 8 + h 4
B_PUSH = 52           # cf[k], cf[rev], cfb[k], cfb[rev] int32 RMW (32) + e(v) int64 RMW (16) + rev 4
B_RELABEL = 4
B_GR_ENTRY = 12       # col 4 + cfb 4 (mirrored reverse residual) + h 4
B_GR_VERTEX = 12      # per vertex per global relabel: h init/finalize, dead, queue
B_RESET = 20          # per slot per solve: cf0 4 + cf 4 + cfb 4 read, cf 4 + cfb 4 written


def algorithmic_bytes(st: dict, n: int, slots: int = 0) -> int:
    """Bytes the method must move in one solve launch, from the kernel's own
    counters; `slots` adds the reset of the residual graph.  An AVQ
    compaction costs B_AVQ_SCAN per vertex when it scans every vertex, and
    the candidate bitmap (n / 8 bytes) plus B_AVQ_SCAN per candidate when it
    works from the bitmap."""
    return (B_ENTRY * st["arcs_scanned"] + B_ACTIVE * st["active_total"] +
            B_AVQ_SCAN * n * st["avq_full_scans"] + (n // 8) * st["avq_bitmap_scans"] +
            B_AVQ_SCAN * st["avq_candidates"] + B_PUSH * st["pushes"] +
            B_RELABEL * st["relabels"] + B_GR_ENTRY * st["gr_arcs_scanned"] +
            B_GR_VERTEX * n * st["global_relabels"] + B_RESET * slots)


def solver_sha() -> str:
    with open(os.path.join(ROOT, "paper_2404_00270_gb300", "csrc", "solver_impl.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profiled_traffic(workload: str):
    """DRAM bytes (read + write) per solve launch from the machine-readable
    ncu record profiles/solve_kernel_<workload>.json, or None when there is
    none or the solver's device code changed since it was captured."""
    try:
        with open(os.path.join(ROOT, "profiles", f"solve_kernel_{workload}.json")) as f:
            rec = json.load(f)
        if not solver_sha().startswith(rec["solver_impl_sha256_prefix"]):
            return None
        return int(rec["dram_bytes_per_launch"])
    except Exception:
        return None


def golden_rmat26():
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_rmat26.json")) as f:
            return json.load(f)
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


def metric_name(workload: str) -> str:
    scale = WORKLOADS[workload]["scale"]
    return f"residual arcs scanned/s (R-MAT {scale} max-flow + min-cut, BCSR)"


def cpu_sample(scale: int = 20, seed: int = 2, cap_hi: int = 1000):
    """The oracle, as it stands, on one host core: one solve (phase 1 +
    phase 2 + edge flows + cut) of the R-MAT `scale` graph."""
    import oracle
    import workloads as W
    oracle.build()
    g = W.rmat(scale, 16, seed, cap_lo=1, cap_hi=cap_hi)
    src, dst, cap = g.numpy()
    t0 = time.perf_counter()
    r = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=True, want_cut=True)
    secs = time.perf_counter() - t0
    return {"value": r["stats"]["arcs_scanned"] / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale {scale} (edge factor 16, seed {seed}, {g.m} arcs; the R-MAT {scale} "
                      f"workload itself), FIFO push-relabel phase 1 + 2 + edge flows + cut, one solve, "
                      f"1 thread; unit = the oracle's own residual arcs examined",
            "time_to_solution_s": secs, "flow_value": r["value"]}


def _oracle_worker_init():
    import oracle  # noqa: F401  (loaded once per worker, before the timed region)


def _oracle_value(inst):
    """The oracle's value (no flow, no cut) of one instance given as
    (n, src, dst, cap, s, t); a task of batch_cpu_baseline's pool."""
    import oracle
    n, src, dst, cap, s, t = inst
    return oracle.maxflow_pr(n, src, dst, cap, s, t, want_flow=False, want_cut=False)["value"]


def batch_cpu_baseline(specs, sample: int) -> dict:
    """The oracle, as it stands, on an evenly spaced sample of the batch mix:
    solves/s on one host core, and with one worker process per host core
    (spawned, so that the pool is safe beside a CUDA context)."""
    import multiprocessing as mp
    import oracle
    import workloads as W
    oracle.build()
    stride = max(1, len(specs) // sample)
    picked = [list(specs[i]) for i in range(0, len(specs), stride)][:sample]
    insts = []
    for sp in picked:
        g = W.make_from_spec(tuple(sp))
        insts.append((g.n, *g.numpy(), g.s, g.t))
    t0 = time.perf_counter()
    for inst in insts:
        _oracle_value(inst)
    one = len(insts) / (time.perf_counter() - t0)
    cores = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_value, insts[:1] * cores, chunksize=1)  # every worker started
        t0 = time.perf_counter()
        pool.map(_oracle_value, insts, chunksize=1)
        allc = len(insts) / (time.perf_counter() - t0)
    return {"value": one, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(picked)} evenly spaced instances of the {len(specs):,}-instance mix (every "
                      f"{stride}th), drawn on the host; FIFO push-relabel, value only; one thread",
            "all_cores": {"value": allc, "unit": "solves/s", "cores": cores,
                          "sample": "the same instances, one worker process per host core (the largest "
                                    "instance bounds the time)"}}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    workload = args.workload if args.workload in WORKLOADS else "rmat26"
    wl = WORKLOADS[workload]
    # each step: the same R-MAT parameters (seed, capacities) at scale 18
    g = W.rmat(18, 16, wl["seed"], cap_lo=1, cap_hi=wl["cap_hi"])
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
    sample = (f"R-MAT scale 18 (edge factor 16, seed {wl['seed']}, capacities U[1,{wl['cap_hi']}], "
              f"{g.m} arcs) per step, a bounded sample of the R-MAT {wl['scale']} workload (same "
              f"generator and parameters, smaller scale); oracle phase 1 + 2 + edge flows + cut, 1 thread")
    # the same workload as the GPU arm's line; each step is the bounded sample above
    config = {"workload": f"{workload}-maxflow-mincut", "scale": wl["scale"], "edge_factor": 16,
              "seed": wl["seed"], "capacities": f"U[1,{wl['cap_hi']}]",
              "parallelism": "replicas" if world > 1 else "single", "sample_per_step": sample}
    line = {"metric": metric_name(workload), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def layout_block(wb, g, stream, layouts, reps: int = 3) -> dict:
    """Per layout, with the graph resident: time to maximum flow (phase 1,
    value only; median of `reps` solves), phase 1 + 2 with edge flows, build
    time, and time to solution (build + maximum flow with edge flows + cut,
    device inputs, host-timed)."""
    import torch
    n, m, s, t = g.n, g.m, g.s, g.t
    flow = torch.empty(max(1, m), dtype=torch.int32, device=g.src.device)
    side = torch.empty(n, dtype=torch.uint8, device=g.src.device)
    out = {}
    for name, layout in layouts:
        torch.cuda.synchronize()
        tb = time.perf_counter()
        G = wb.wbpr_build(n, m, g.src, g.dst, g.cap, s, t, layout, None, stream)
        torch.cuda.synchronize()
        build_ms = 1e3 * (time.perf_counter() - tb)
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
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G = wb.wbpr_build(n, m, g.src, g.dst, g.cap, s, t, layout, None, stream)
        v = wb.wbpr_maxflow(G, stream, flow)
        c = wb.wbpr_mincut(G, stream, side)
        G.close()
        torch.cuda.synchronize()
        tts_ms = 1e3 * (time.perf_counter() - t0)
        assert len(set(vals)) == 1 and vals[0] == v == c
        out[name] = {"value": vals[0], "time_to_maxflow_ms": statistics.median(t_ms),
                     "arcs_per_s": statistics.median(arcs_l) / (statistics.median(t_ms) / 1e3),
                     "build_ms": build_ms, "phase1_plus_phase2_ms": st2["solve_ms"],
                     "time_to_solution_ms": tts_ms,
                     "iterations": st2["iterations"], "global_relabels": st2["global_relabels"],
                     "device_bytes": info["device_bytes"], "slots": info["slots"],
                     "grid_blocks": info["grid_blocks"], "renumbered": bool(info["renumbered"])}
    return out


def run_gpu(args):
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

    wl = WORKLOADS[args.workload]
    g = W.rmat(wl["scale"], 16, wl["seed"], cap_lo=1, cap_hi=wl["cap_hi"], device=dev)
    n, m, s, t = g.n, g.m, g.s, g.t
    flow = torch.empty(m, dtype=torch.int32, device=dev)
    side = torch.empty(n, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    opts = None
    if args.options:
        opts = wb.wbpr_default_options()
        for k, v in json.loads(args.options).items():
            setattr(opts, k, v)

    def step():
        G = wb.wbpr_build(n, m, g.src, g.dst, g.cap, s, t, wb.WBPR_BCSR, opts, stream)
        v = wb.wbpr_maxflow(G, stream, flow)
        st = wb.wbpr_get_stats(G)
        c = wb.wbpr_mincut(G, stream, side)
        info = wb.wbpr_get_info(G)
        G.close()
        return v, c, st, info

    for _ in range(max(1, args.warmup)):
        v0, c0, _, info0 = step()
    assert v0 == c0

    torch.cuda.reset_peak_memory_stats(dev)
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
        v, c, st, info = step()
        arcs += st["arcs_scanned"]
        solve_ms += st["solve_ms"]
        alg_bytes += algorithmic_bytes(st, n, info["slots"])
        value_seen = v
        assert v == c == v0
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    peak_bytes = torch.cuda.max_memory_allocated(dev)
    ms = ev0.elapsed_time(ev1)
    ms, arcs_all = aggregate_ranks(ms, float(arcs), dev)
    value = arcs_all / (ms / 1e3)

    # the headline graph resident (BCSR), and R-MAT 20 in both layouts
    headline = {} if args.quick else layout_block(wb, g, stream, [("bcsr", wb.WBPR_BCSR)])
    c2 = {}
    if not args.quick:
        if args.workload == "rmat20":
            c2 = layout_block(wb, g, stream, [("bcsr", wb.WBPR_BCSR), ("rcsr", wb.WBPR_RCSR)])
        else:
            g20 = W.rmat(20, 16, 2, device=dev)
            c2 = layout_block(wb, g20, stream, [("bcsr", wb.WBPR_BCSR), ("rcsr", wb.WBPR_RCSR)])
            c2["workload"] = f"rmat20 (n {g20.n}, m {g20.m}, seed 2, capacities U[1,1000])"
            del g20
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e_steps = 0 if args.quick else max(1, min(args.steps, 3))
    e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 12 * m, "d2h_bytes_per_step": 4 * m + n + 16}
    if e_steps:
        hsrc = g.src.cpu().pin_memory()
        hdst = g.dst.cpu().pin_memory()
        hcap = g.cap.cpu().pin_memory()
        hflow = torch.empty(m, dtype=torch.int32).pin_memory()
        hside = torch.empty(n, dtype=torch.uint8).pin_memory()
        # one untimed step first: the library's staging buffers for host
        # inputs and outputs come from the caching allocator on first use
        G = wb.wbpr_build(n, m, hsrc, hdst, hcap, s, t, wb.WBPR_BCSR, None, stream)
        wb.wbpr_maxflow(G, stream, hflow)
        wb.wbpr_mincut(G, stream, hside)
        G.close()
        barrier()
        t0 = time.perf_counter()
        e_arcs = 0
        for _ in range(e_steps):
            G = wb.wbpr_build(n, m, hsrc, hdst, hcap, s, t, wb.WBPR_BCSR, None, stream)
            ve = wb.wbpr_maxflow(G, stream, hflow)
            e_arcs += wb.wbpr_get_stats(G)["arcs_scanned"]
            ce = wb.wbpr_mincut(G, stream, hside)
            G.close()
            assert ve == ce == value_seen
        barrier()
        e_ms = 1e3 * (time.perf_counter() - t0)
        e_ms, e_arcs_all = aggregate_ranks(e_ms, float(e_arcs), dev)
        e2e["value"] = e_arcs_all / (e_ms / 1e3)
        e2e["ms_per_step"] = e_ms / e_steps
        del hsrc, hdst, hcap, hflow, hside

    peak, peak_kind = measured_peaks()
    launch_ms = solve_ms / args.steps
    achieved = (alg_bytes / args.steps) / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.workload)
    footprint = {"handle_bytes": info0["device_bytes"], "peak_device_bytes_in_step": peak_bytes,
                 "coo_bytes": 12 * m, "adjacency_matrix_bytes_2B_per_cell": 2 * n * n,
                 "matrix_over_handle": 2 * n * n / info0["device_bytes"]}
    config = {"workload": f"{args.workload}-maxflow-mincut", "scale": wl["scale"], "edge_factor": 16,
              "seed": wl["seed"], "capacities": f"U[1,{wl['cap_hi']}]", "n": n, "m": m, "s": s, "t": t,
              "layout": "bcsr+rev", "renumbered": bool(info0["renumbered"]),
              "parallelism": "replicas" if world > 1 else "single",
              "l2": f"inputs larger than L2 (COO {12 * m / 1e6:.0f} MB, BCSR handle "
                    f"{info0['device_bytes'] / 1e6:.0f} MB per step); no flush needed",
              "flow_value": value_seen, "options": json.loads(args.options) if args.options else {},
              "time_to_maxflow_ms": headline["bcsr"]["time_to_maxflow_ms"] if headline else None,
              "resident": headline, "footprint": footprint, "layouts_rmat20": c2}
    gold = golden_rmat26() if args.workload == "rmat26" else None
    if gold:
        config["oracle_offline"] = {"value": gold["value"], "equal": gold["value"] == value_seen,
                                    "wall_s": gold["oracle_wall_s"], "host": gold["host"],
                                    "source": "tests/golden/oracle_rmat26.json"}
    line = {
        "metric": metric_name(args.workload), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "solve_kernel",
                     "launch_ms": launch_ms, "algorithmic_bytes_per_launch": alg_bytes / args.steps,
                     "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})"},
        "gpu_launches": args.steps * launches_per_step(bool(info0["renumbered"]), m),
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_sample(20, 2, 1000)
        if c2:
            gpu_tts = c2["bcsr"]["time_to_solution_ms"] / 1e3
            cb["gpu_time_to_solution_s"] = gpu_tts
            cb["speedup_time_to_solution"] = cb["time_to_solution_s"] / gpu_tts
            assert cb["flow_value"] == c2["bcsr"]["value"]
        line["cpu_baseline"] = cb
    if rank == 0 and world == 1 and not args.quick and args.batch_block > 0:
        line["config"]["batch"] = batch_measure(args.batch_block, steps=3, warmup=1, plain_sample=24,
                                                serve_count=args.batch_block, serve_rates=[1.0])
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()

def batch_measure(count: int, steps: int, warmup: int, plain_sample: int, serve_count: int,
                  serve_rates, tune: bool = False) -> dict:
    """The batched / served workload: `count` instances of the seeded mix of
    grids and bipartite graphs of uneven size, solved (a) one instance per
    launch on an evenly spaced sample, (b) all in one batched launch per step,
    (c) through the continuous-batching server with Poisson arrivals at
    fractions of the batched rate.  Every batched and served value must equal
    the one-at-a-time value of the same instance (the oracle checks of the
    whole mix are in tests/test_gpu_c5_mix.py).  With `tune`, the batch knobs are tuned per graph class (autotune.tune_batch),
    the batched launch is timed again with every handle set to its class's
    options, and the served runs use them too."""
    import numpy as np
    import torch
    import paper_2404_00270_gb300 as wb
    from paper_2404_00270_gb300 import serve
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    wb.load()
    wb.use_torch_allocator(True)
    stream = torch.cuda.current_stream()
    specs = W.batch_spec(count)
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
    stride = max(1, len(graphs) // plain_sample)
    sample = list(range(0, len(graphs), stride))
    plain_ms, plain_vals = [], {}
    for i in sample:
        torch.cuda.synchronize()
        ta = time.perf_counter()
        plain_vals[i] = wb.wbpr_maxflow(graphs[i], stream)
        plain_ms.append(1e3 * (time.perf_counter() - ta))
    plain_rate = len(sample) / (sum(plain_ms) / 1e3)

    # (b) the whole mix in one batched launch per step
    for _ in range(warmup):
        vals = wb.wbpr_maxflow_batch(graphs, stream)
    assert all(vals[i] == plain_vals[i] for i in sample)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        vals = wb.wbpr_maxflow_batch(graphs, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    assert all(vals[i] == plain_vals[i] for i in sample)
    batch_rate = len(graphs) / (ms / 1e3)
    tuned = {}
    table = None
    if tune:
        from paper_2404_00270_gb300 import autotune
        t0 = time.perf_counter()
        table = autotune.tune_batch(insts, stream=stream)
        tuned["tune_s"] = time.perf_counter() - t0
        tuned["classes"] = len(table.entries)
        autotune.apply_table(graphs, table)
        vals_t = wb.wbpr_maxflow_batch(graphs, stream)
        assert list(vals_t) == list(vals)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            vals_t = wb.wbpr_maxflow_batch(graphs, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        tuned["batched_solves_per_s"] = len(graphs) / (ev0.elapsed_time(ev1) / steps / 1e3)
        tuned["speedup_vs_default_batch"] = tuned["batched_solves_per_s"] / batch_rate
    inst_ms = [wb.wbpr_get_stats(G)["solve_ms"] for G in graphs]
    slowest = sorted(range(len(graphs)), key=lambda i: -inst_ms[i])[:5]
    slowest = [{"spec": list(specs[i]), "ms": inst_ms[i], "team_blocks": wb.wbpr_get_info(graphs[i])["grid_blocks"]}
               for i in slowest]
    batch_vals = list(vals)
    for G in graphs:
        G.close()
    del graphs
    torch.cuda.empty_cache()
    # (c) continuous batching with Poisson arrivals at a fraction of the batch rate
    serving = {}
    rng = np.random.default_rng(5)
    n_serve = min(len(insts), serve_count)
    for frac in serve_rates:
        lam = frac * batch_rate
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_serve))
        reqs = [serve.Request(i, g.n, g.src, g.dst, g.cap, g.s, g.t, float(a))
                for i, (g, a) in enumerate(zip(insts[:n_serve], arrivals))]
        free_b, _ = torch.cuda.mem_get_info()
        srv = serve.Server(int(0.5 * free_b), table=table)
        out = srv.run(reqs)
        bad = [r.rid for r in out if r.value != batch_vals[r.rid]]
        assert not bad, bad
        summ = serve.latency_summary(out)
        summ["rate_per_s"] = lam
        serving[f"{frac:g}x"] = summ
    return {"instances": len(insts), "arcs": total_arcs, "generate_s": gen_s, "build_s": build_s,
            "layout": "bcsr+rev", "batched_solves_per_s": batch_rate, "batch_ms": ms,
            "plain_solves_per_s": plain_rate, "plain_sample": len(sample),
            "plain_p50_ms": float(np.percentile(plain_ms, 50)),
            "plain_p99_ms": float(np.percentile(plain_ms, 99)),
            "speedup_vs_plain": batch_rate / plain_rate,
            "tuned": tuned, "slowest_in_batch": slowest, "serving": serving}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    res = batch_measure(args.batch_count, args.steps, args.warmup, args.plain_sample, args.serve_count,
                        args.serve_rates, tune=args.tune)
    clocks = sampler.stop()
    cpu = None
    if args.oracle_sample > 0:
        import workloads as W
        cpu = batch_cpu_baseline(W.batch_spec(args.batch_count), args.oracle_sample)
    line = {
        "metric": f"batched solves/s ({res['instances']:,}-instance mix, one batched launch)",
        "value": res["batched_solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["batch_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(res, workload=f"batch-mix-{res['instances']}"),
        "roofline": None, "clocks": clocks, "gpu_launches": args.steps * 2,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))


def warp_distribution(w) -> dict:
    """Per-warp busy times normalised by their mean (the distribution of
    §4.3, Fig. 3): spread and quantiles."""
    import numpy as np
    w = np.asarray(w, np.float64)
    if w.size == 0 or w.mean() <= 0:
        return {}
    x = w / w.mean()
    return {"warps": int(w.size), "mean_us": float(w.mean() / 1e3), "std_over_mean": float(x.std()),
            "max_over_mean": float(x.max()),
            "quantiles_over_mean": {f"p{q}": float(np.percentile(x, q)) for q in (5, 25, 50, 75, 95)}}


def run_ablation(args):
    """Vertex-centric (VC, the method) against thread-centric (TC, the
    lock-free baseline of Alg. 1): the comparison of the paper's Tables 1-2
    and Fig. 3 on the R-MAT 20 and bipartite 2^20 workloads, both layouts,
    with the discharge pass and with the paper's one-push rule.  Per
    configuration: time to maximum flow (phase 1, median of up to 3 solves;
    one when a solve takes over 2 s), iterations, and the per-warp busy-time
    distribution."""
    import torch
    import paper_2404_00270_gb300 as wb
    import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wb.load()
    wb.use_torch_allocator(True)
    stream = torch.cuda.current_stream()
    graphs = {"rmat20": lambda: W.rmat(20, 16, 2, device=dev),
              "bipartite20": lambda: W.bipartite_zipf(1 << 20, 1 << 20, 3, device=dev)}
    rows = []
    for gname, make in graphs.items():
        g = make()
        for lname, layout in (("bcsr", wb.WBPR_BCSR), ("rcsr", wb.WBPR_RCSR)):
            for mp in (1, 0):
                for tc in (0, 1):
                    o = wb.wbpr_default_options()
                    o.thread_centric, o.multi_push, o.warp_time = tc, mp, 1
                    G = wb.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, layout, o, stream)
                    times, vals = [], []
                    for _ in range(3):
                        vals.append(wb.wbpr_maxflow(G, stream))
                        st = wb.wbpr_get_stats(G)
                        times.append(st["solve_ms"])
                        if st["solve_ms"] > 2000:
                            break
                    w = wb.wbpr_export(G, "warp_time")
                    G.close()
                    assert len(set(vals)) == 1
                    rows.append({"graph": gname, "layout": lname, "approach": "TC" if tc else "VC",
                                 "push_rule": "discharge pass" if mp else "one push (Alg. 1)",
                                 "value": vals[0], "time_to_maxflow_ms": statistics.median(times),
                                 "iterations": st["iterations"], "arcs_scanned": st["arcs_scanned"],
                                 "warps": warp_distribution(w)})
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del g
        torch.cuda.empty_cache()
    speedups = {}
    for r in rows:
        if r["approach"] == "VC":
            tcr = next(x for x in rows if x["approach"] == "TC" and all(
                x[k] == r[k] for k in ("graph", "layout", "push_rule")))
            assert tcr["value"] == r["value"]
            speedups[f"{r['graph']}/{r['layout']}/{r['push_rule']}"] = tcr["time_to_maxflow_ms"] / r["time_to_maxflow_ms"]
    line = {"metric": "time to maximum flow, thread-centric / vertex-centric (speedup of VC)",
            "value": statistics.mean(speedups.values()), "unit": "x", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "ablation-vc-tc", "speedups": speedups, "rows": rows}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wbpr", choices=["wbpr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="timed steps only (profiling runs)")
    ap.add_argument("--workload", default="rmat26", choices=["rmat26", "rmat22", "rmat20", "batch", "ablation"])
    ap.add_argument("--batch-block", type=int, default=256,
                    help="instances of the batch / serving block in config (0 = none)")
    ap.add_argument("--batch-count", type=int, default=1024)
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--serve-count", type=int, default=512)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[0.5, 1.0])
    ap.add_argument("--tune", action="store_true", help="batch: per-class tuned knobs, timed again")
    ap.add_argument("--oracle-sample", type=int, default=32,
                    help="batch: instances of the mix the CPU oracle solves for cpu_baseline (0 = none)")
    ap.add_argument("--options", default="",
                    help='library options of the timed handle as JSON, e.g. {"thread_centric": 1} (profiling)')
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "ablation":
        run_ablation(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
