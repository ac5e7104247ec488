"""Multi-source / multi-sink instances (the construction of §4.1): a super
source S* feeds every source s_i and every sink t_i drains into a super sink
T*, each super arc carrying the total capacity at its terminal.  Pinned on
the CPU against facts that do not depend on the construction's code: one
pair gives the plain s-t maximum flow, k disjoint paths give the sum of
their bottlenecks, more pairs never give less flow, and the oracle's
push-relabel agrees with Dinic and with cut enumeration."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W


def _value(g):
    src, dst, cap = g.numpy()
    return oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=False, want_cut=False)["value"]


def test_structure():
    g = W.random_small(10, 40, 3, cap_lo=1)
    mt = W.multi_terminal(g, [0, 1], [7, 8])
    assert mt.n == g.n + 2 and mt.m == g.m + 4 and (mt.s, mt.t) == (g.n, g.n + 1)
    src, dst, cap = (x.numpy().astype(np.int64) for x in (g.src, g.dst, g.cap))
    msrc, mdst, mcap = (x.numpy() for x in (mt.src, mt.dst, mt.cap))
    assert np.array_equal(msrc[:g.m], src) and np.array_equal(mdst[:g.m], dst)
    assert list(msrc[g.m:g.m + 2]) == [g.n, g.n] and list(mdst[g.m:g.m + 2]) == [0, 1]
    assert list(mdst[g.m + 2:]) == [g.n + 1, g.n + 1] and list(msrc[g.m + 2:]) == [7, 8]
    assert mcap[g.m] == cap[src == 0].sum() and mcap[g.m + 1] == cap[src == 1].sum()
    assert mcap[g.m + 2] == cap[dst == 7].sum() and mcap[g.m + 3] == cap[dst == 8].sum()
    with pytest.raises(ValueError):
        W.multi_terminal(g, [0, 1], [1, 2])


@pytest.mark.parametrize("seed", range(40))
def test_one_pair_is_the_plain_maxflow(seed):
    g = W.random_small(9, 30, seed, cap_lo=0, cap_hi=9)
    mt = W.multi_terminal(g, [g.s], [g.t])
    src, dst, cap = mt.numpy()
    v = _value(mt)
    assert v == _value(g)
    assert v == oracle.mincut_brute(mt.n, src, dst, cap, mt.s, mt.t)[0]


def test_disjoint_paths_sum_of_bottlenecks():
    # k disjoint paths s_i -> a_i -> b_i -> t_i with capacities (c1, c2, c3)
    rng = np.random.default_rng(7)
    src, dst, cap, sources, sinks = [], [], [], [], []
    total = 0
    for i in range(6):
        base = 4 * i
        c = rng.integers(1, 50, size=3)
        src += [base, base + 1, base + 2]
        dst += [base + 1, base + 2, base + 3]
        cap += list(c)
        sources.append(base)
        sinks.append(base + 3)
        total += int(c.min())
    g = W.FlowInstance("paths", 24, torch.tensor(src, dtype=torch.int32), torch.tensor(dst, dtype=torch.int32),
                       torch.tensor(cap, dtype=torch.int32), 0, 3)
    assert _value(W.multi_terminal(g, sources, sinks)) == total


def test_rmat_multi_pairs_monotone_and_dinic():
    g = W.rmat_multi(10, 8, 3, 4)
    src_s, snk = g.meta["sources"], g.meta["sinks"]
    assert len(src_s) == 4 and not set(src_s) & set(snk)
    src, dst, cap = g.numpy()
    v = _value(g)
    assert v > 0 and v == oracle.maxflow_dinic(g.n, src, dst, cap, g.s, g.t)["value"]
    base = W.rmat(10, 8, 3)
    prev = 0
    for k in range(1, 5):
        vk = _value(W.multi_terminal(base, src_s[:k], snk[:k]))
        assert vk >= prev
        prev = vk
    assert prev == v
