"""The CPU oracle against values fixed by the paper's definitions and by
mathematics (hand-computed fixtures, enumeration of every cut, closed forms,
Dinic, Hopcroft-Karp, the Koenig certificate)."""
import numpy as np
import pytest

from tests import oracle_pins as P


def test_golden_fixtures(oracle_mod):
    P.pin_golden()


def test_verifier_rejects_broken_flows(oracle_mod):
    P.pin_verifier()


def test_residual_distances(oracle_mod):
    P.pin_residual_dist()


def test_residual_distances_match_library_shortest_paths(oracle_mod):
    """The global-relabel heights of a residual snapshot (Section 2.2: the
    exact distance to the sink over arcs with positive residual capacity,
    never through the source) against SciPy's unweighted shortest paths on
    the reversed graph with the source's arcs removed: an independent
    breadth-first search on random arc lists with loops, duplicates and zero
    residuals."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    import oracle
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(2, 200))
        na = int(rng.integers(0, 6 * n))
        tail = rng.integers(0, n, na).astype(np.int32)
        head = rng.integers(0, n, na).astype(np.int32)
        res = rng.integers(-1, 4, na).astype(np.int64)
        target = int(rng.integers(0, n))
        excluded = int(rng.integers(0, n)) if trial % 3 else -1
        if excluded == target:
            excluded = -1
        base, unreach, excl_h = int(trial % 5), n + 7, n + 3
        got = oracle.residual_dist(n, tail, head, res, target, excluded, base, unreach, excl_h)
        keep = res > 0
        if excluded >= 0:
            keep &= (tail != excluded) & (head != excluded)
        # reversed arcs head -> tail, so distances from the target are
        # distances to it in the residual graph
        a = sp.csr_matrix((np.ones(int(keep.sum())), (head[keep], tail[keep])), shape=(n, n))
        d = csgraph.shortest_path(a, method="D", directed=True, unweighted=True, indices=target)
        want = np.where(np.isfinite(d), base + np.nan_to_num(d, posinf=0).astype(np.int64), unreach)
        if excluded >= 0:
            want[excluded] = excl_h
        assert got.tolist() == want.tolist(), (trial, n, na)


def test_value_and_cut_side_match_scipy_maximum_flow(oracle_mod):
    pytest.importorskip("scipy.sparse.csgraph")
    P.pin_library_maxflow()


def test_closed_forms(oracle_mod):
    P.pin_closed_forms()


def test_bruteforce_cuts(oracle_mod):
    P.pin_bruteforce(count=1500)


def test_matching_vs_hopcroft_karp(oracle_mod):
    P.pin_matching()


def test_dinic_agreement_medium(oracle_mod):
    import workloads as W
    for seed in range(12):
        n = 50 + 37 * seed
        inst = W.random_small(n, 6 * n, 100 + seed, cap_lo=0, cap_hi=50 + seed)
        src, dst, cap = inst.numpy()
        args = (n, src, dst, cap, inst.s, inst.t)
        pr = oracle_mod.maxflow_pr(*args)
        di = oracle_mod.maxflow_dinic(*args, want_flow=True)
        assert pr["value"] == di["value"]
        code, cut, side = oracle_mod.verify_flow(*args, pr["flow"], pr["value"])
        assert code == 0 and cut == pr["value"]
        # Both maximum flows give the same canonical cut side.
        code2, _, side2 = oracle_mod.verify_flow(*args, di["flow"], di["value"])
        assert code2 == 0 and (side == side2).all()
        assert (side == pr["source_side"]).all()


def test_grid_c1_value_is_stable(oracle_mod):
    """The 64x64 grid with U[1,100] capacities, seed 1 (value written by
    tests/golden/make_golden.py from the oracle, cross-checked by Dinic)."""
    import json, os
    import workloads as W
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_values.json")))
    g = W.grid(64, 64, 1)
    src, dst, cap = g.numpy()
    v = oracle_mod.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    assert v == gold["grid64x64_seed1"]
    assert oracle_mod.maxflow_dinic(g.n, src, dst, cap, g.s, g.t)["value"] == v


def test_invalid_inputs(oracle_mod):
    with pytest.raises(RuntimeError):
        oracle_mod.maxflow_pr(3, [0], [1], [1], 0, 0)         # s == t
    with pytest.raises(RuntimeError):
        oracle_mod.maxflow_pr(3, [0], [5], [1], 0, 1)         # id out of range
    with pytest.raises(RuntimeError):
        oracle_mod.maxflow_pr(3, [0], [1], [-1], 0, 1)        # negative capacity
