"""The thread-centric (TC) baseline and the per-warp time record, through
the C ABI.

TC (wbpr_options.thread_centric = 1) is the lock-free push-relabel of Alg. 1
as the paper's TC+RCSR / TC+BCSR rows run it: one thread per vertex, no
active-vertex queue, each active vertex's list scanned by its own thread.
It must give the oracle's results like the vertex-centric path: value, cut
capacity and canonical cut side bit-exact, edge flows certified, with the
discharge pass and with the paper's one-push rule, in both layouts.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_helpers import LAYOUTS, check_against_oracle, gpu_solve, wb

pytestmark = pytest.mark.gpu


def _opts(m, **kw):
    o = m.wbpr_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("multi_push", [1, 0])
@pytest.mark.parametrize("layout", LAYOUTS)
def test_tc_kernel_matches_oracle(layout, multi_push):
    m = wb()
    o = _opts(m, thread_centric=1, multi_push=multi_push)
    for seed in range(80):
        n = 2 + seed % 14
        inst = W.random_small(n, (seed * 5) % 48, 9600 + seed, cap_lo=0 if seed % 3 else 1, cap_hi=1 + seed % 17)
        src, dst, cap = inst.numpy()
        bv, bs = oracle.mincut_brute(n, src, dst, cap, inst.s, inst.t)
        got = gpu_solve(n, src, dst, cap, inst.s, inst.t, layout, o)
        assert got["value"] == bv == got["cut"], seed
        assert np.array_equal(got["side"], bs), seed
        assert oracle.verify_flow(n, src, dst, cap, inst.s, inst.t, got["flow"], bv)[0] == 0, seed
    graphs = [W.rmat(12, 16, 5), W.grid(32, 32, 6), W.bipartite_zipf(2048, 2048, 7)]
    if multi_push:
        graphs.append(W.rmat(14, 16, 2))
    for g in graphs:
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o)


@pytest.mark.parametrize("thread_centric", [0, 1])
def test_warp_time_record(thread_centric):
    """Every warp of the grid gets a busy time; the record does not change
    the result and is off by default."""
    m = wb()
    g = W.bipartite_zipf(4096, 4096, 3)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_RCSR,
                     _opts(m, thread_centric=thread_centric, warp_time=1))
    assert m.wbpr_maxflow(G) == ref
    info = m.wbpr_get_info(G)
    w = m.wbpr_export(G, "warp_time")
    assert w.size == 8 * info["grid_blocks"]
    assert w.sum() > 0
    st = m.wbpr_get_stats(G)
    assert w.max() < 1e6 * max(1.0, st["solve_ms"]) * 1.5   # no warp is busy longer than the launch
    G.close()
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_RCSR)
    assert m.wbpr_maxflow(G) == ref
    assert m.wbpr_export(G, "warp_time").size == 0
    G.close()
