"""The pins that tie the oracle to the paper and to mathematics.

Each function raises AssertionError on a mismatch.  They are shared by
``test_oracle.py`` and by ``test_oracle_mutations.py``, which checks that a
deliberately broken oracle fails at least one of them.
"""
import numpy as np

import oracle
import workloads as W
from tests.golden import FIXTURES, load


def pin_golden():
    """Hand-computed fixtures (tests/golden/*.txt)."""
    for name in FIXTURES:
        f = load(name)
        args = (f["n"], f["src"], f["dst"], f["cap"], f["s"], f["t"])
        pr = oracle.maxflow_pr(*args)
        assert pr["value"] == f["value"], (name, pr["value"])
        assert (pr["source_side"] == f["source_side"]).all(), name
        assert oracle.maxflow_dinic(*args)["value"] == f["value"], name
        bv, bs = oracle.mincut_brute(*args)
        assert bv == f["value"] and (bs == f["source_side"]).all(), name
        code, cut, side = oracle.verify_flow(*args, pr["flow"], pr["value"])
        assert code == 0 and cut == f["value"] and (side == f["source_side"]).all(), name


def pin_bruteforce(count=600, seed0=0):
    """Every s-t cut enumerated on random graphs of <= 13 vertices."""
    for seed in range(seed0, seed0 + count):
        n = 2 + seed % 12
        m = (seed * 7) % 41
        lo = 0 if seed % 3 else 1
        inst = W.random_small(n, m, seed, cap_lo=lo, cap_hi=1 + seed % 17)
        src, dst, cap = inst.numpy()
        args = (n, src, dst, cap, inst.s, inst.t)
        pr = oracle.maxflow_pr(*args)
        bv, bs = oracle.mincut_brute(*args)
        assert pr["value"] == bv, (seed, pr["value"], bv)
        assert (pr["source_side"] == bs).all(), seed
        code, cut, _ = oracle.verify_flow(*args, pr["flow"], pr["value"])
        assert code == 0 and cut == bv, (seed, code)
        assert oracle.maxflow_dinic(*args)["value"] == bv, seed


def pin_closed_forms():
    # R x C grid with uniform capacity c <= terminal capacity: R disjoint
    # row paths of bottleneck c, and the cut after column 0 has capacity R*c.
    for (r, c, cc) in [(3, 4, 7), (8, 5, 50), (16, 16, 1), (64, 64, 50)]:
        g = W.grid(r, c, 1, uniform_cap=cc)
        src, dst, cap = g.numpy()
        assert oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"] == r * cc
    # A path 0 -> 1 -> ... -> k has value = its smallest capacity.
    rng = np.random.default_rng(5)
    for k in (1, 2, 5, 40):
        caps = rng.integers(1, 1000, size=k).astype(np.int32)
        src = np.arange(k, dtype=np.int32)
        dst = src + 1
        assert oracle.maxflow_pr(k + 1, src, dst, caps, 0, k)["value"] == caps.min()
    # Complete bipartite K_{a,b} with unit arcs: value min(a, b).
    for a, b in [(1, 1), (3, 5), (7, 2), (20, 20)]:
        s, t = a + b, a + b + 1
        src, dst = [], []
        for i in range(a):
            for j in range(b):
                src.append(i); dst.append(a + j)
        src += [s] * a + list(range(a, a + b))
        dst += list(range(a)) + [t] * b
        cap = np.ones(len(src), np.int32)
        assert oracle.maxflow_pr(a + b + 2, src, dst, cap, s, t)["value"] == min(a, b)
    # A planted perfect matching plus random extra edges: value = nl.
    nl = 300
    perm = rng.permutation(nl)
    eu = list(range(nl)) + list(rng.integers(0, nl, 900))
    ev = list(perm) + list(rng.integers(0, nl, 900))
    s, t = 2 * nl, 2 * nl + 1
    src = eu + [s] * nl + list(range(nl, 2 * nl))
    dst = [nl + v for v in ev] + list(range(nl)) + [t] * nl
    cap = np.ones(len(src), np.int32)
    assert oracle.maxflow_pr(2 * nl + 2, src, dst, cap, s, t)["value"] == nl
    # Disjoint s-t paths: the value is the sum of their bottlenecks.
    src, dst, cap = [], [], []
    total, nxt = 0, 2
    for L in (1, 2, 3, 7):
        cs = rng.integers(1, 100, size=L + 1)
        prev = 0
        for j in range(L):
            src.append(prev); dst.append(nxt); cap.append(cs[j]); prev = nxt; nxt += 1
        src.append(prev); dst.append(1); cap.append(cs[L])
        total += int(cs.min())
    assert oracle.maxflow_pr(nxt, src, dst, np.array(cap, np.int32), 0, 1)["value"] == total
    # A single arc; a reversed single arc.
    assert oracle.maxflow_pr(2, [0], [1], [17], 0, 1)["value"] == 17
    assert oracle.maxflow_pr(2, [1], [0], [17], 0, 1)["value"] == 0


def _bip_network(nl, nr, eu, ev):
    s, t = nl + nr, nl + nr + 1
    src = list(eu) + [s] * nl + list(range(nl, nl + nr))
    dst = [nl + v for v in ev] + list(range(nl)) + [t] * nr
    return nl + nr + 2, np.array(src, np.int32), np.array(dst, np.int32), \
        np.ones(len(src), np.int32), s, t


def pin_matching(count=60):
    """Hopcroft-Karp size = max-flow value; Koenig vertex cover certificate."""
    rng = np.random.default_rng(11)
    for it in range(count):
        nl, nr = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        ne = int(rng.integers(0, 4 * (nl + nr)))
        eu = rng.integers(0, nl, ne)
        ev = rng.integers(0, nr, ne)
        hk = oracle.matching_hk(nl, nr, eu, ev)
        n, src, dst, cap, s, t = _bip_network(nl, nr, eu, ev)
        pr = oracle.maxflow_pr(n, src, dst, cap, s, t)
        assert pr["value"] == hk, (it, pr["value"], hk)
        Z = pr["source_side"].astype(bool)
        # Koenig: (L \ Z) u (R n Z) covers every edge and has size = matching.
        cover_l = ~Z[:nl]
        cover_r = Z[nl:nl + nr]
        assert int(cover_l.sum() + cover_r.sum()) == hk
        for u, v in zip(eu, ev):
            assert cover_l[u] or cover_r[v]


def pin_verifier():
    """The certificate check rejects each kind of broken flow."""
    f = load("diamond.txt")
    args = (f["n"], f["src"], f["dst"], f["cap"], f["s"], f["t"])
    pr = oracle.maxflow_pr(*args)
    flow = pr["flow"].copy()
    assert oracle.verify_flow(*args, flow, 5)[0] == 0
    bad = flow.copy(); bad[0] = f["cap"][0] + 1
    assert oracle.verify_flow(*args, bad, 5)[0] == 1          # over capacity
    bad = flow.copy(); bad[0] = -1
    assert oracle.verify_flow(*args, bad, 5)[0] == 1          # negative
    bad = flow.copy(); bad[2] += 1 if bad[2] < f["cap"][2] else -1
    assert oracle.verify_flow(*args, bad, 5)[0] == 2          # conservation
    assert oracle.verify_flow(*args, flow, 4)[0] == 3         # wrong value
    # A valid but non-maximum flow: 0-2-3 carries 2 units only.
    small = np.zeros_like(flow)
    small[1] = 2; small[4] = 2
    assert oracle.verify_flow(*args, small, 2)[0] == 4


def pin_residual_dist():
    """Backward BFS distances on a hand-made residual arc list."""
    # arcs: 0->1, 1->2, 2->3, 0->3 (residual 0), 4->0, 5 isolated
    tail = [0, 1, 2, 0, 4]
    head = [1, 2, 3, 3, 0]
    res = [1, 1, 1, 0, 2]
    d = oracle.residual_dist(6, tail, head, res, 3, 5, 0, 6, 6)
    assert list(d) == [3, 2, 1, 0, 4, 6]
    d = oracle.residual_dist(6, tail, head, res, 3, 1, 10, 99, 7)
    assert list(d) == [99, 7, 11, 10, 99, 99]


def _scipy_maxflow(n, src, dst, cap, s, t):
    """SciPy's maximum flow (its own Dinic) on the same arcs: parallel arcs
    merge by summing their capacities, self-loops are dropped (they carry no
    flow).  Returns the value and the minimal source side: the vertices
    reachable from s over arcs with residual capacity c(u, v) - f(u, v) > 0,
    where f is SciPy's antisymmetric flow."""
    import scipy.sparse as sp
    from scipy.sparse import csgraph
    keep = src != dst
    c = sp.csr_matrix((cap[keep].astype(np.int64), (src[keep], dst[keep])), shape=(n, n)).astype(np.int32)
    res = csgraph.maximum_flow(c, s, t, method="dinic")
    resid = (c.tocsr() - res.flow.tocsr()).tocsr()   # c(u, v) - f(u, v); f(v, u) = -f(u, v)
    resid.data = np.maximum(resid.data, 0)
    resid.eliminate_zeros()
    order = csgraph.breadth_first_order(resid, s, directed=True, return_predecessors=False)
    side = np.zeros(n, np.uint8)
    side[order] = 1
    assert side[s] == 1 and side[t] == 0
    return int(res.flow_value), side


def pin_library_maxflow():
    """The oracle's value and canonical source side S* against SciPy's
    maximum_flow, an implementation written independently of this one, on
    random graphs with loops, duplicates, antiparallel pairs and zero
    capacities, and on small R-MAT and bipartite workloads.  S* is the same
    for every maximum flow (the intersection of all minimum source sides),
    so it must agree bit for bit."""
    rng = np.random.default_rng(5)
    cases = []
    for trial in range(40):
        n = int(rng.integers(3, 400))
        m = int(rng.integers(0, 8 * n))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        cap = rng.integers(0, 1000, m).astype(np.int32)
        s, t = rng.choice(n, 2, replace=False)
        cases.append((n, src, dst, cap, int(s), int(t)))
    for g in (W.rmat(12, 16, 7, cap_lo=1, cap_hi=1000), W.bipartite_zipf(2048, 2048, 3)):
        cases.append((g.n, *g.numpy(), g.s, g.t))
    for n, src, dst, cap, s, t in cases:
        r = oracle.maxflow_pr(n, src, dst, cap, s, t, want_flow=False, want_cut=True)
        value, side = _scipy_maxflow(n, src, dst, cap, s, t)
        assert r["value"] == value, (n, src.size)
        assert r["source_side"].tolist() == side.tolist(), (n, src.size)


ALL_PINS = [pin_golden, pin_verifier, pin_residual_dist, pin_closed_forms,
            pin_bruteforce, pin_matching, pin_library_maxflow]
