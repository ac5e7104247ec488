"""Oracle values of seeded batch-mix instances, computed in worker
processes (multiprocessing with spawn, safe after CUDA is in use).  Each
worker draws its instance on the CPU from the spec and runs the oracle's
push-relabel on it.  Test infrastructure only."""
import multiprocessing as mp
import os


def spec_value(spec):
    import oracle
    import workloads as W
    g = W.make_from_spec(tuple(spec))
    src, dst, cap = g.numpy()
    return oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=False, want_cut=False)["value"]


def spec_values(specs, procs=None):
    import oracle
    oracle.build()   # once, before the workers load it
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(spec_value, [list(s) for s in specs], chunksize=1)
