"""Renumbered handles and paper-mode BCSR, through the C ABI.

* Renumbering (wbpr_options.renumber = 1): the builder gives the vertices
  new ids by endpoint count, largest first, and solves on those.  Every
  result must still be the oracle's in input ids: flow value, cut capacity
  and canonical cut side bit-exact, edge flows certified.  The layout the
  handle holds must be, array for array, the layout of §3.2 of the
  relabelled graph (the oracle's by-definition restatement applied to the
  relabelled arcs), and the order must be the stated one.
* Paper-mode BCSR (use_rev = 0 at build time): the backward slot is found by
  binary search in the neighbour's sorted row (§3.2), so the handle holds
  neither the reverse index nor the mirrored reverse residual: exactly 8
  bytes per slot less, with the same results.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import layouts
from tests.gpu_helpers import LAYOUTS, check_against_oracle, gpu_solve, layout_code, wb

pytestmark = pytest.mark.gpu


def _opts(m, **kw):
    o = m.wbpr_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("layout", LAYOUTS)
def test_renumbered_small_vs_bruteforce(layout):
    m = wb()
    o = _opts(m, renumber=1)
    for seed in range(120):
        n = 2 + seed % 14
        inst = W.random_small(n, (seed * 7) % 48, 9300 + seed, cap_lo=0 if seed % 3 else 1, cap_hi=1 + seed % 19)
        src, dst, cap = inst.numpy()
        bv, bs = oracle.mincut_brute(n, src, dst, cap, inst.s, inst.t)
        got = gpu_solve(n, src, dst, cap, inst.s, inst.t, layout, o)
        assert got["value"] == bv == got["cut"], seed
        assert np.array_equal(got["side"], bs), seed
        assert oracle.verify_flow(n, src, dst, cap, inst.s, inst.t, got["flow"], bv)[0] == 0, seed


@pytest.mark.parametrize("layout", LAYOUTS)
def test_renumbered_matches_oracle(layout):
    m = wb()
    o = _opts(m, renumber=1)
    for g in (W.rmat(14, 16, 2), W.bipartite_zipf(4096, 4096, 3), W.grid(64, 64, 1), W.rmat_multi(12, 16, 5, 4)):
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_renumbered_layout_is_the_relabelled_graph(layout):
    m = wb()
    inst = W.random_small(300, 3000, 77, cap_lo=0, cap_hi=1000)
    src, dst, cap = inst.numpy()
    src = np.concatenate([src, src[:100], dst[100:300], [5, 9]]).astype(np.int32)
    dst = np.concatenate([dst, dst[:100], src[100:300], [5, 9]]).astype(np.int32)
    cap = np.concatenate([cap, cap[:100], cap[100:300], [3, 4]]).astype(np.int32)
    n = inst.n
    G = m.wbpr_build(n, src.size, src, dst, cap, inst.s, inst.t, layout_code(layout), _opts(m, renumber=1))
    assert m.wbpr_get_info(G)["renumbered"] == 1
    order = m.wbpr_export(G, "order")
    # endpoint counts of the non-loop arcs, largest first, ties by input id
    loop = src == dst
    deg = np.bincount(src[~loop], minlength=n) + np.bincount(dst[~loop], minlength=n)
    assert np.array_equal(order, np.lexsort((np.arange(n), -deg)))
    perm = np.empty(n, np.int64)
    perm[order] = np.arange(n)
    assert m.wbpr_export(G, "st").tolist() == [perm[inst.s], perm[inst.t]]
    rs, rd = perm[src].astype(np.int32), perm[dst].astype(np.int32)
    ref = layouts.bcsr(n, rs, rd, cap) if layout == "bcsr" else layouts.rcsr(n, rs, rd, cap)
    for key, val in ref.items():
        assert np.array_equal(m.wbpr_export(G, key), val), key
    G.close()


def test_input_numbering_exports_no_order():
    m = wb()
    g = W.grid(8, 8, 1)
    src, dst, cap = g.numpy()
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR, _opts(m, renumber=0))
    assert m.wbpr_get_info(G)["renumbered"] == 0
    assert m.wbpr_export(G, "order").size == 0
    assert m.wbpr_export(G, "st").tolist() == [g.s, g.t]
    o = m.wbpr_get_options(G)
    o.renumber = 1
    with pytest.raises(m.WbprError) as e:
        m.wbpr_set_options(G, o)
    assert e.value.status == -6
    G.close()


def test_paper_mode_bcsr_holds_no_reverse_index():
    m = wb()
    for g in (W.rmat(14, 16, 2), W.bipartite_zipf(4096, 4096, 3), W.grid(48, 48, 2)):
        src, dst, cap = g.numpy()
        G1 = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR)
        G0 = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR, _opts(m, use_rev=0))
        i1, i0 = m.wbpr_get_info(G1), m.wbpr_get_info(G0)
        assert i1["slots"] == i0["slots"] > 0
        assert i1["device_bytes"] - i0["device_bytes"] == 8 * i1["slots"]
        with pytest.raises(m.WbprError):
            m.wbpr_export(G0, "rev")
        o = m.wbpr_get_options(G0)
        o.use_rev = 1
        with pytest.raises(m.WbprError) as e:
            m.wbpr_set_options(G0, o)
        assert e.value.status == -6
        G1.close()
        G0.close()


@pytest.mark.parametrize("bu", [(0, 1024, 1), (14, 1024, 1), (1 << 20, 1, 0)])
def test_paper_mode_bcsr_matches_oracle(bu):
    """Binary-search backward lookup in the push, the global relabel and
    the cut BFS, top-down, switched, or bottom-up."""
    m = wb()
    o = _opts(m, use_rev=0, bottom_up=bu[0], bottom_up_min=bu[1], bottom_up_edges=bu[2])
    for g in (W.rmat(14, 16, 41), W.bipartite_zipf(4096, 4096, 43), W.grid(40, 40, 47)):
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, "bcsr", o)
