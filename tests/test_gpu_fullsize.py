"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (default options).

* R-MAT scale 20 (16.1 M arcs), both layouts, and the bipartite 2^20 x 2^20
  matching network: flow value, cut capacity and canonical cut side equal
  the oracle's, the matching size equals Hopcroft-Karp's, and every edge
  flow passes the optimality certificate.
* R-MAT scale 26 (1.06 G arcs): the oracle's push-relabel takes about 18
  minutes on one host core there, so it ran once, offline
  (tests/golden/make_golden.py), and its value, the SHA-256 of its packed
  canonical cut side and the SHA-256 of the input arrays are stored in
  tests/golden/oracle_rmat26.json.  The GPU must draw the same graph and
  give that value and that cut side; on top of that, the certificate holds
  at any size: capacity and conservation of every edge flow, and a residual
  cut whose capacity equals the flow value (so the flow is maximum), plus
  the GPU's cut side equal to the one the certificate computes.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import layout_code, wb

pytestmark = pytest.mark.gpu


def _solve(g, layout, renumber=-1):
    m = wb()
    o = m.wbpr_default_options()
    o.renumber = renumber
    G = m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, layout_code(layout), o)
    flow = torch.empty(g.m, dtype=torch.int32, device=g.src.device)
    side = torch.empty(g.n, dtype=torch.uint8, device=g.src.device)
    value = m.wbpr_maxflow(G, None, flow)
    cut = m.wbpr_mincut(G, None, side)
    G.close()
    return value, cut, flow.cpu().numpy(), side.cpu().numpy()


@pytest.fixture(scope="module")
def rmat20():
    g = W.rmat(20, 16, 2, device="cuda:0")
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=False, want_cut=True)
    return g, ref


@pytest.mark.parametrize("renumber", [0, 1])
@pytest.mark.parametrize("layout", ["bcsr", "rcsr"])
def test_rmat20_full(rmat20, layout, renumber):
    g, ref = rmat20
    value, cut, flow, side = _solve(g, layout, renumber)
    assert value == ref["value"] == cut
    assert np.array_equal(side, ref["source_side"])
    src, dst, cap = g.numpy()
    code, c2, _ = oracle.verify_flow(g.n, src, dst, cap, g.s, g.t, flow, value)
    assert code == 0 and c2 == value


def test_bipartite20_full():
    g = W.bipartite_zipf(1 << 20, 1 << 20, 3, device="cuda:0")
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, want_flow=False, want_cut=True)
    lr, nl = g.meta["lr_edges"], g.meta["nl"]
    hk = oracle.matching_hk(nl, g.meta["nr"], src[:lr], dst[:lr] - nl)
    value, cut, flow, side = _solve(g, "bcsr")
    assert value == ref["value"] == hk == cut
    assert np.array_equal(side, ref["source_side"])
    code, c2, _ = oracle.verify_flow(g.n, src, dst, cap, g.s, g.t, flow, value)
    assert code == 0 and c2 == value


@pytest.mark.slow
def test_rmat26_certificate():
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 180 * (1 << 30):
        pytest.skip("needs about 180 GB of free device memory")
    g = W.rmat(26, 16, 4, cap_lo=1, cap_hi=10000, device="cuda:0")
    m = wb()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_rmat26.json")))
    assert (g.n, g.m, g.s, g.t) == (gold["n"], gold["m"], gold["s"], gold["t"])
    G = m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, layout_code("bcsr"))
    from bench import algorithmic_bytes
    for _ in range(2):   # phase 1 only, for the record (run with -s to see it)
        v1 = m.wbpr_maxflow(G)
        st = m.wbpr_get_stats(G)
        ab = algorithmic_bytes(st, g.n, m.wbpr_get_info(G)["slots"])
        print(f"R-MAT 26 phase 1: value {v1}, {st['solve_ms']:.1f} ms, {st['iterations']} iterations, "
              f"{st['global_relabels']} global relabels, algorithmic bytes {ab / 1e9:.1f} GB "
              f"({ab / (st['solve_ms'] * 1e6):.0f} GB/s), handle {m.wbpr_get_info(G)['device_bytes'] / 1e9:.1f} GB")
    G.close()
    value, cut, flow, side = _solve(g, "bcsr")
    assert value == cut == v1 == gold["value"]
    assert int(np.count_nonzero(side)) == gold["source_side_count"]
    assert hashlib.sha256(np.packbits(side != 0).tobytes()).hexdigest() == gold["source_side_sha256"]
    n, s, t = g.n, g.s, g.t
    src, dst, cap = g.numpy()
    del g
    torch.cuda.empty_cache()
    h = hashlib.sha256()
    for a in (src, dst, cap):
        for lo in range(0, a.size, 1 << 26):
            h.update(a[lo:lo + (1 << 26)].tobytes())
    assert h.hexdigest() == gold["graph_sha256"]   # the graph the oracle solved
    code, c2, S = oracle.verify_flow(n, src, dst, cap, s, t, flow, value)
    assert code == 0 and c2 == value
    assert np.array_equal(S, side)
