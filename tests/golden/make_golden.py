"""Writes the stored oracle values under tests/golden/ from the CPU oracle only.

Run from the repository root:

    python tests/golden/make_golden.py
        oracle_values.json: values of three small seeded workloads (seconds).

    python tests/golden/make_golden.py --rmat26 --scratch DIR
        oracle_rmat26.json: the massive R-MAT workload (scale 26, edge factor
        16, seed 4, capacities U[1, 10^4]; 1.07 G arcs).  The graph is drawn
        once in a child process and written to DIR as .npy files, so that the
        oracle process holds only its own residual graph (about 53 GB) while
        the inputs stay memory-mapped.  Drawing the graph on the CPU took
        about 12 minutes, the oracle's FIFO push-relabel on one host core
        (phase 1, phase 2 and the cut BFS) about 18 (oracle_wall_s records
        it).  Stored: the maximum-flow value, a SHA-256 of the packed
        canonical source side S* (np.packbits, bit order big), |S*|, and a
        SHA-256 of the input arrays so that a test can check that it draws
        the same graph.

    python tests/golden/make_golden.py --rmat26 --dinic --scratch DIR
        adds Dinic's value for the same graph (from the arrays in DIR) to
        oracle_rmat26.json, an independent cross-check of the stored value.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402

RMAT26 = dict(scale=26, edge_factor=16, seed=4, cap_lo=1, cap_hi=10000)


def graph_sha256(src, dst, cap) -> str:
    h = hashlib.sha256()
    for a in (src, dst, cap):
        a = np.ascontiguousarray(a, dtype=np.int32)
        step = 1 << 26
        for lo in range(0, a.size, step):
            h.update(a[lo:lo + step].tobytes())
    return h.hexdigest()


def side_sha256(side) -> str:
    return hashlib.sha256(np.packbits(np.asarray(side, np.uint8) != 0).tobytes()).hexdigest()


def small():
    out = {}
    g = W.grid(64, 64, 1)
    src, dst, cap = g.numpy()
    out["grid64x64_seed1"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    g = W.rmat(14, 16, 2)
    src, dst, cap = g.numpy()
    out["rmat14_seed2"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    g = W.bipartite_zipf(1 << 12, 1 << 12, 3)
    src, dst, cap = g.numpy()
    out["bipartite4096_seed3"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    with open(os.path.join(HERE, "oracle_values.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(out)


def _draw_rmat26(scratch):
    g = W.rmat(RMAT26["scale"], RMAT26["edge_factor"], RMAT26["seed"],
               cap_lo=RMAT26["cap_lo"], cap_hi=RMAT26["cap_hi"])
    src, dst, cap = g.numpy()
    for name, a in (("src", src), ("dst", dst), ("cap", cap)):
        np.save(os.path.join(scratch, name + ".npy"), a)
    with open(os.path.join(scratch, "meta.json"), "w") as f:
        json.dump({"n": g.n, "m": g.m, "s": g.s, "t": g.t}, f)


def rmat26(scratch):
    os.makedirs(scratch, exist_ok=True)
    t0 = time.time()
    if not os.path.exists(os.path.join(scratch, "meta.json")):
        p = mp.get_context("spawn").Process(target=_draw_rmat26, args=(scratch,))
        p.start()
        p.join()
        if p.exitcode != 0:
            raise SystemExit("drawing the graph failed")
    with open(os.path.join(scratch, "meta.json")) as f:
        meta = json.load(f)
    src, dst, cap = (np.load(os.path.join(scratch, k + ".npy"), mmap_mode="r") for k in ("src", "dst", "cap"))
    t_gen = time.time() - t0
    gsha = graph_sha256(src, dst, cap)
    print(f"graph n={meta['n']} m={meta['m']} s={meta['s']} t={meta['t']} sha256={gsha} ({t_gen:.0f} s)", flush=True)
    t1 = time.time()
    ref = oracle.maxflow_pr(meta["n"], src, dst, cap, meta["s"], meta["t"], want_flow=False, want_cut=True)
    t_oracle = time.time() - t1
    side = ref["source_side"]
    out = {
        "workload": "rmat26_seed4_cap1-10000",
        "params": RMAT26,
        "n": meta["n"], "m": meta["m"], "s": meta["s"], "t": meta["t"],
        "graph_sha256": gsha,
        "value": int(ref["value"]),
        "source_side_count": int(np.count_nonzero(side)),
        "source_side_sha256": side_sha256(side),
        "oracle": "oracle_maxflow_pr (FIFO push-relabel, phase 1 + phase 2 + cut BFS), one thread",
        "oracle_stats": {k: int(v) for k, v in ref["stats"].items()},
        "oracle_wall_s": round(t_oracle, 1),
        "host": {"machine": platform.machine(), "cpu": _cpu_model(), "cores_used": 1,
                 "cores_available": os.cpu_count()},
    }
    with open(os.path.join(HERE, "oracle_rmat26.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


def rmat26_dinic(scratch):
    """Cross-check of the stored R-MAT 26 value with Dinic's algorithm, on
    the same drawn arrays (their SHA-256 must match the stored one)."""
    path = os.path.join(HERE, "oracle_rmat26.json")
    with open(path) as f:
        out = json.load(f)
    with open(os.path.join(scratch, "meta.json")) as f:
        meta = json.load(f)
    src, dst, cap = (np.load(os.path.join(scratch, k + ".npy"), mmap_mode="r") for k in ("src", "dst", "cap"))
    if graph_sha256(src, dst, cap) != out["graph_sha256"]:
        raise SystemExit("the drawn arrays are not the stored graph")
    t0 = time.time()
    ref = oracle.maxflow_dinic(meta["n"], src, dst, cap, meta["s"], meta["t"])
    out["dinic_value"] = int(ref["value"])
    out["dinic_wall_s"] = round(time.time() - t0, 1)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rmat26", action="store_true")
    ap.add_argument("--dinic", action="store_true",
                    help="with --rmat26: add Dinic's value for the stored graph (drawn arrays reused)")
    ap.add_argument("--scratch", default=None, help="directory for the drawn R-MAT 26 arrays")
    a = ap.parse_args()
    if a.rmat26:
        if not a.scratch:
            raise SystemExit("--rmat26 needs --scratch DIR")
        oracle.build()
        if a.dinic:
            rmat26_dinic(a.scratch)
        else:
            rmat26(a.scratch)
    else:
        small()


if __name__ == "__main__":
    main()
