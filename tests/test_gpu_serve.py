"""Continuous batching: every request's result is the same alone and in the
mix, while requests arrive during other solves (the persistent server kernel
picks each one up as soon as a team of its size class is free) and admission
is limited by a device-memory budget."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import wb

pytestmark = pytest.mark.gpu


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    insts = []
    for i in range(count):
        k = i % 4
        if k == 0:
            insts.append(W.grid(int(rng.integers(8, 40)), int(rng.integers(8, 40)), 300 + i, 1, 255, 2550))
        elif k == 1:
            insts.append(W.bipartite_poisson(int(rng.integers(50, 800)), int(rng.integers(50, 800)),
                                             int(rng.integers(4, 17)), 400 + i))
        elif k == 2:
            insts.append(W.rmat(int(rng.integers(8, 12)), 8, 500 + i))
        else:
            insts.append(W.random_small(int(rng.integers(20, 300)), int(rng.integers(50, 2000)), 600 + i,
                                        cap_lo=0, cap_hi=50))
    return insts


def test_served_results_equal_alone():
    m = wb()
    from paper_2404_00270_gb300 import serve
    insts = _mix(48, 7)
    dev = torch.device("cuda:0")
    # alone: one solve per instance
    alone = []
    for g in insts:
        src, dst, cap = g.numpy()
        G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR)
        alone.append(m.wbpr_maxflow(G))
        G.close()
        assert alone[-1] == oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
    rng = np.random.default_rng(3)
    arrivals = np.cumsum(rng.exponential(0.002, size=len(insts)))
    reqs = []
    for i, (g, a) in enumerate(zip(insts, arrivals)):
        d = g.to(dev)
        reqs.append(serve.Request(i, g.n, d.src, d.dst, d.cap, g.s, g.t, float(a)))
    budget = 4 * max(serve.footprint_estimate(r.n, r.m) for r in reqs)
    srv = serve.Server(budget, big_slots=4000, team_blocks=4, big_teams=8, small_blocks=64)
    out = srv.run(reqs)
    assert [r.value for r in out] == alone
    assert all(r.done >= r.admitted >= r.arrival for r in out)
    # admission was limited by the budget: never more than it in flight at once
    assert srv.peak_in_use <= budget + max(r.footprint for r in out)
    summ = serve.latency_summary(out)
    assert summ["solves"] == len(insts) and summ["p99_ms"] >= summ["p50_ms"] > 0
    # the solves overlapped on the device: some were in progress at the same time
    assert all(r.device_ns and r.device_ns[1] >= r.device_ns[0] for r in out)
    assert summ["max_concurrent_on_device"] >= 2
