"""CUDA path vs the oracle, through the C ABI.  Integer work: every compared
quantity (flow value, cut capacity, canonical cut side, builder arrays,
preflow state, global-relabel heights) must match bit for bit; edge flows
are not unique and are checked by the optimality certificate."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import layouts
from tests.golden import FIXTURES, load
from tests.gpu_helpers import LAYOUTS, check_against_oracle, gpu_solve, layout_code, wb

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("name", FIXTURES)
def test_golden_fixtures(name, layout):
    f = load(name)
    got = check_against_oracle(f["n"], f["src"], f["dst"], f["cap"], f["s"], f["t"], layout)
    assert got["value"] == f["value"]
    assert np.array_equal(got["side"], f["source_side"])


@pytest.mark.parametrize("layout", LAYOUTS)
def test_random_small_vs_bruteforce(layout):
    for seed in range(300):
        n = 2 + seed % 14
        m = (seed * 5) % 48
        inst = W.random_small(n, m, 7000 + seed, cap_lo=0 if seed % 3 else 1, cap_hi=1 + seed % 23)
        src, dst, cap = inst.numpy()
        bv, bs = oracle.mincut_brute(n, src, dst, cap, inst.s, inst.t)
        got = gpu_solve(n, src, dst, cap, inst.s, inst.t, layout)
        assert got["value"] == bv == got["cut"], (seed, got["value"], bv)
        assert np.array_equal(got["side"], bs), seed
        code, _, _ = oracle.verify_flow(n, src, dst, cap, inst.s, inst.t, got["flow"], bv)
        assert code == 0, (seed, code)


def test_bcsr_binary_search_mode_matches():
    m = wb()
    o = m.wbpr_default_options()
    o.use_rev = 0
    for seed in range(40):
        inst = W.random_small(30 + seed, 200, 9100 + seed, cap_lo=0, cap_hi=40)
        src, dst, cap = inst.numpy()
        check_against_oracle(inst.n, src, dst, cap, inst.s, inst.t, "bcsr", o)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_grid_64x64(layout):
    g = W.grid(64, 64, 1)
    src, dst, cap = g.numpy()
    got = check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout)
    assert got["value"] == 1971


@pytest.mark.parametrize("layout", LAYOUTS)
def test_grid_uniform_closed_form(layout):
    g = W.grid(64, 64, 1, uniform_cap=50)
    src, dst, cap = g.numpy()
    got = gpu_solve(g.n, src, dst, cap, g.s, g.t, layout)
    assert got["value"] == 64 * 50


@pytest.mark.parametrize("layout", LAYOUTS)
def test_medium_random_with_duplicates(layout):
    for seed in range(6):
        n = 500 + 300 * seed
        inst = W.random_small(n, 8 * n, 500 + seed, cap_lo=0, cap_hi=100)
        src, dst, cap = inst.numpy()
        # duplicate a slice of arcs and reverse another slice (antiparallel pairs)
        src = np.concatenate([src, src[:200], dst[200:400]])
        dst = np.concatenate([dst, dst[:200], src[200:400]])
        cap = np.concatenate([cap, cap[:200], cap[200:400]])
        check_against_oracle(n, src, dst, cap, inst.s, inst.t, layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_rmat_14(layout):
    g = W.rmat(14, 16, 2)
    src, dst, cap = g.numpy()
    got = check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout)
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_values.json")))
    assert got["value"] == gold["rmat14_seed2"]


@pytest.mark.parametrize("layout", LAYOUTS)
def test_bipartite_matching(layout):
    g = W.bipartite_zipf(1 << 12, 1 << 12, 3)
    src, dst, cap = g.numpy()
    got = check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout)
    lr = g.meta["lr_edges"]
    nl = g.meta["nl"]
    hk = oracle.matching_hk(nl, g.meta["nr"], src[:lr], dst[:lr] - nl)
    assert got["value"] == hk


@pytest.mark.parametrize("multi_push", [1, 0])
def test_option_sweep_same_results(multi_push):
    m = wb()
    g = W.rmat(12, 16, 5)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)
    for layout in LAYOUTS:
        for tile, smax, wmax, gap, cycle, grid in [(4, 4, 64, 1, 1, 0), (16, 16, 16, 0, 1000, 0),
                                                   (8, 0, 0, 1, 7, 3), (8, 8, 2048, 1, 64, 1)]:
            o = m.wbpr_default_options()
            o.small_tile, o.small_max_degree, o.warp_max_degree = tile, smax, wmax
            o.gap, o.cycle, o.grid_blocks, o.multi_push = gap, cycle, grid, multi_push
            check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o, ref=ref)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("multi_push", [1, 0])
def test_incremental_avq_same_results(layout, multi_push):
    """AVQ compactions built from the candidate bitmap between global
    relabels (avq_incremental = 1), block-local passes for small AVQs on top
    of that (2, the default) and full scans of every vertex (0) all give the
    oracle's value, cut side and a certified flow, with the gap heuristic on
    and off and with short and long relabel cycles (many incremental
    compactions and local passes in a row)."""
    m = wb()
    graphs = [W.rmat(12, 16, 5), W.grid(40, 40, 3), W.random_small(300, 3000, 77, cap_lo=0, cap_hi=50)]
    for g in graphs:
        src, dst, cap = g.numpy()
        ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)
        for inc, gap, cycle, ratio in [(2, 1, 0, 1.5), (2, 0, 0, 1.5), (2, 1, 1000, 0.0), (2, 0, 50, 0.0),
                                       (1, 1, 0, 1.5), (1, 0, 1000, 0.0), (0, 1, 0, 1.5)]:
            o = m.wbpr_default_options()
            o.multi_push, o.avq_incremental, o.gap, o.cycle, o.gr_ratio = multi_push, inc, gap, cycle, ratio
            st = check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o, ref=ref)["stats"]
            # every iteration compacts its AVQ one way or the other; a full
            # scan follows every global relabel; no bitmap without the option
            assert st["avq_full_scans"] + st["avq_bitmap_scans"] >= st["iterations"]
            assert st["avq_full_scans"] >= 1
            if not inc:
                assert st["avq_bitmap_scans"] == 0 and st["avq_candidates"] == 0


@pytest.mark.parametrize("layout", LAYOUTS)
def test_single_push_mode_small_graphs(layout):
    """The one-push-per-iteration rule of Alg. 1/2 gives the same results."""
    m = wb()
    o = m.wbpr_default_options()
    o.multi_push = 0
    for seed in range(60):
        n = 2 + seed % 14
        inst = W.random_small(n, (seed * 5) % 48, 8000 + seed, cap_lo=0, cap_hi=9)
        src, dst, cap = inst.numpy()
        bv, bs = oracle.mincut_brute(n, src, dst, cap, inst.s, inst.t)
        got = gpu_solve(n, src, dst, cap, inst.s, inst.t, layout, o)
        assert got["value"] == bv and np.array_equal(got["side"], bs), seed
        assert oracle.verify_flow(n, src, dst, cap, inst.s, inst.t, got["flow"], bv)[0] == 0


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("lean", [0, 1])
def test_builder_arrays_bit_exact(layout, lean):
    """Every builder array equals the by-definition layout, with duplicate,
    antiparallel and self-loop arcs, for CUB's tuning and for lean builds
    (256-thread sort blocks, duplicate prefixes by run), on inputs past and
    within the single-tile size of the sorts."""
    m = wb()
    o = m.wbpr_default_options()
    o.lean_build = lean
    for seed in range(5):
        inst = W.random_small(200 + 50 * seed, 3000 if seed < 4 else 400, 300 + seed, cap_lo=0, cap_hi=1000)
        src, dst, cap = inst.numpy()
        src = np.concatenate([src, src[:100], dst[100:300], [5, 9]])
        dst = np.concatenate([dst, dst[:100], src[100:300], [5, 9]])
        cap = np.concatenate([cap, cap[:100], cap[100:300], [3, 4]])
        G = m.wbpr_build(inst.n, src.size, src, dst, cap, inst.s, inst.t, layout_code(layout), o)
        ref = layouts.bcsr(inst.n, src, dst, cap) if layout == "bcsr" else layouts.rcsr(inst.n, src, dst, cap)
        for key, val in ref.items():
            got = m.wbpr_export(G, key)
            assert np.array_equal(got, val), (layout, key)
        G.close()


# (bottom_up, bottom_up_min, bottom_up_edges)
BU_MODES = {"top-down": (0, 1024, 1), "default": (14, 1024, 1), "vertex-rule": (14, 1024, 0),
            "phase-aware": (14, 1024, 2), "bottom-up": (1 << 20, 1, 0)}


def _bu_options(m, mode):
    o = m.wbpr_default_options()
    o.bottom_up, o.bottom_up_min, o.bottom_up_edges = BU_MODES[mode]
    return o


@pytest.mark.parametrize("bu", list(BU_MODES))
@pytest.mark.parametrize("layout", LAYOUTS)
def test_preflow_and_global_relabel_stages(layout, bu):
    """Preflow state and global-relabel heights (BFS distances to t over the
    residual arcs of the exported snapshot, s excluded) bit-exact, with the
    BFS levels top-down, bottom-up, or switched by frontier size."""
    m = wb()
    g = W.rmat(11, 8, 9)
    src, dst, cap = g.numpy()
    n, s, t = g.n, g.s, g.t
    G = m.wbpr_build(n, src.size, src, dst, cap, s, t, layout_code(layout), _bu_options(m, bu))
    m.wbpr_run_stage(G, 1)   # preflow
    h = m.wbpr_export(G, "height")
    e = m.wbpr_export(G, "excess")
    exp_h = np.zeros(n, np.int32)
    exp_h[s] = n
    assert np.array_equal(h, exp_h)
    exp_e = np.zeros(n, np.int64)
    np.add.at(exp_e, dst[src == s], cap[src == s].astype(np.int64))
    exp_e[s] = 0
    loops = (src == s) & (dst == s)
    assert not loops.any()
    assert np.array_equal(e, exp_e)
    assert m.wbpr_export(G, "excess_total")[0] == cap[src == s].sum()
    for rounds in (0, 3, 25):
        if rounds:
            m.wbpr_run_stage(G, 3, rounds)   # push-relabel iterations, no relabel
        m.wbpr_run_stage(G, 2)               # one global relabel
        tail, head, res = _residual_arcs(m, G, n, layout)
        dist = oracle.residual_dist(n, tail, head, res, t, s, 0, n, n)
        h = m.wbpr_export(G, "height")
        alive = dist < n
        assert np.array_equal(h[alive], dist[alive]), rounds
        assert (h[~alive] >= n).all()
    G.close()


def _residual_arcs(m, G, n, layout):
    off = m.wbpr_export(G, "offsets")
    col = m.wbpr_export(G, "col")
    cf = m.wbpr_export(G, "cf").astype(np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(off))
    if layout == "bcsr":
        return rows, col, cf
    bf = m.wbpr_export(G, "bf").astype(np.int64)
    # forward residual u -> v = cf, backward residual v -> u = bf
    return np.concatenate([rows, col]), np.concatenate([col, rows]), np.concatenate([cf, bf])


def test_resolve_is_idempotent():
    m = wb()
    g = W.grid(32, 32, 3)
    src, dst, cap = g.numpy()
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR)
    a = m.wbpr_maxflow(G)
    b = m.wbpr_maxflow(G)
    flow = np.zeros(g.m, np.int32)   # host buffer: copied back by the library
    c = m.wbpr_maxflow(G, None, flow)
    assert a == b == c
    assert oracle.verify_flow(g.n, src, dst, cap, g.s, g.t, flow, c)[0] == 0
    G.close()


def test_pinned_host_buffers_match_oracle():
    """Inputs and outputs in page-locked host memory: the flows and the cut
    side are written by the kernels straight into the mapped host buffers,
    and equal the oracle's results (value, cut side, certified flow)."""
    m = wb()
    g = W.rmat(12, 16, 9)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)
    hs, hd, hc = (torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (src, dst, cap))
    for layout in LAYOUTS:
        G = m.wbpr_build(g.n, g.m, hs, hd, hc, g.s, g.t, layout_code(layout))
        flow = torch.full((g.m,), -7, dtype=torch.int32).pin_memory()
        side = torch.full((g.n,), 9, dtype=torch.uint8).pin_memory()
        v = m.wbpr_maxflow(G, None, flow)
        c = m.wbpr_mincut(G, None, side)
        G.close()
        assert v == c == ref["value"], layout
        assert np.array_equal(side.numpy(), ref["source_side"]), layout
        assert oracle.verify_flow(g.n, src, dst, cap, g.s, g.t, flow.numpy(), v)[0] == 0, layout


def test_iteration_cap_reports_timeout_and_handle_survives():
    m = wb()
    g = W.grid(32, 32, 4)
    src, dst, cap = g.numpy()
    o = m.wbpr_default_options()
    o.max_iterations = 2
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR, o)
    with pytest.raises(m.WbprError) as e:
        m.wbpr_maxflow(G)
    assert e.value.status == -4
    o.max_iterations = 1 << 40
    m.wbpr_set_options(G, o)
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    assert m.wbpr_maxflow(G) == ref
    G.close()


def test_device_errors_are_reported():
    m = wb()
    with pytest.raises(m.WbprError) as e:
        m.wbpr_build(10, 2, [0, 1], [1, 11], [1, 1], 0, 9)    # id out of range
    assert e.value.status == -1
    with pytest.raises(m.WbprError) as e:
        m.wbpr_build(10, 1, [0], [1], [-1], 0, 9)              # negative capacity
    assert e.value.status == -1
    big = 2 ** 31 - 1
    with pytest.raises(m.WbprError) as e:
        m.wbpr_build(4, 2, [0, 1], [1, 0], [big, 5], 0, 3)     # pair sum overflows int32
    assert e.value.status == -5


def test_degenerate_graphs():
    for layout in LAYOUTS:
        # no arcs at all; only self-loops; s -> t directly
        got = gpu_solve(2, [], [], [], 0, 1, layout)
        assert got["value"] == 0 and got["side"].tolist() == [1, 0]
        got = gpu_solve(3, [0, 1, 2], [0, 1, 2], [5, 5, 5], 0, 2, layout)
        assert got["value"] == 0 and got["flow"].tolist() == [0, 0, 0]
        got = gpu_solve(2, [0, 0, 1], [1, 1, 0], [5, 7, 3], 0, 1, layout)
        assert got["value"] == 12 and got["flow"].tolist() == [5, 7, 0]


def _batch_instances():
    out = []
    for seed in range(12):
        out.append(W.random_small(20 + 13 * seed, 150 + 40 * seed, 4200 + seed, cap_lo=0, cap_hi=30))
    for side in (8, 16, 33):
        out.append(W.grid(side, side, 50 + side, 1, 255, 2550))
    for nl in (64, 300):
        out.append(W.bipartite_poisson(nl, nl, 6, 70 + nl))
    out.append(W.rmat(11, 16, 9))
    out.append(W.rmat(12, 8, 10))
    return out


@pytest.mark.parametrize("big_slots", [1 << 20, 3000])
def test_batch_matches_oracle(big_slots):
    """One batched launch (single-block solves, and teams of blocks for the
    instances above `batch_big_slots`) gives every instance its own maximum
    flow, the same as solving it alone; edge flows are certified."""
    m = wb()
    insts = _batch_instances()
    o = m.wbpr_default_options()
    o.batch_big_slots = big_slots
    o.batch_team = 8
    graphs, flows, refs = [], [], []
    for i, inst in enumerate(insts):
        src, dst, cap = inst.numpy()
        layout = m.WBPR_BCSR if i % 2 == 0 else m.WBPR_RCSR
        graphs.append(m.wbpr_build(inst.n, inst.m, src, dst, cap, inst.s, inst.t, layout, o))
        flows.append(torch.empty(max(1, inst.m), dtype=torch.int32, device="cuda:0") if i % 3 == 0 else None)
        refs.append(oracle.maxflow_pr(inst.n, src, dst, cap, inst.s, inst.t, want_flow=False, want_cut=False)["value"])
    values = m.wbpr_maxflow_batch(graphs, None, flows)
    assert values == refs
    for i, inst in enumerate(insts):
        if flows[i] is not None:
            src, dst, cap = inst.numpy()
            code, cut, _ = oracle.verify_flow(inst.n, src, dst, cap, inst.s, inst.t,
                                              flows[i][: inst.m].cpu().numpy(), values[i])
            assert code == 0 and cut == refs[i], (i, code)
    # a second batch on the same handles (state reused) and single solves agree
    assert m.wbpr_maxflow_batch(graphs) == refs
    assert [m.wbpr_maxflow(G) for G in graphs[:5]] == refs[:5]
    for G in graphs:
        G.close()


@pytest.mark.parametrize("ratio", [0.0, 0.25, 1.0, 8.0])
def test_time_balanced_relabel_same_results(ratio):
    m = wb()
    o = m.wbpr_default_options()
    o.gr_ratio = ratio
    for g in (W.rmat(12, 16, 21), W.grid(24, 24, 5)):
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, "bcsr", o)


@pytest.mark.parametrize("bu", list(BU_MODES))
@pytest.mark.parametrize("layout", LAYOUTS)
def test_bottom_up_bfs_same_results(layout, bu):
    """Value, cut and canonical side do not depend on the BFS direction, on
    graphs whose middle levels are large (R-MAT, bipartite) and on a grid
    (long thin levels); hub rows are scanned by whole blocks bottom-up."""
    m = wb()
    o = _bu_options(m, bu)
    for g in (W.rmat(14, 16, 41), W.bipartite_zipf(4096, 4096, 43), W.grid(40, 40, 47)):
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o)
    o.warp_max_degree = 16   # rows over 16 entries scanned by whole blocks
    g = W.rmat(12, 16, 45)
    src, dst, cap = g.numpy()
    check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout, o)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_multi_source_rmat(layout):
    """Eight far-apart source / sink pairs on R-MAT 13, joined by a super
    source and a super sink (the multi-terminal construction of §4.1)."""
    g = W.rmat_multi(13, 16, 5, 8)
    src, dst, cap = g.numpy()
    check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout)


def test_autotune_keeps_the_value():
    from paper_2404_00270_gb300 import autotune
    m = wb()
    g = W.rmat(11, 16, 33)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
    cfg, ms, trials = autotune.autotune(g.n, g.m, src, dst, cap, g.s, g.t, limit=12, reps=1)
    assert len(trials) == 12 and ms > 0
    o = m.wbpr_default_options()
    for k, v in cfg.items():
        setattr(o, k, v)
    check_against_oracle(g.n, src, dst, cap, g.s, g.t, "bcsr", o)


@pytest.mark.parametrize("warp_max", [16, 1024])
def test_staged_hub_chunks_same_results(warp_max):
    """Hub rows read through the shared-memory stage (stage_hubs = 1), with
    many hubs (rows over 16 entries) or the default class bounds."""
    m = wb()
    o = m.wbpr_default_options()
    o.stage_hubs = 1
    o.warp_max_degree = warp_max
    o.small_max_degree = min(8, warp_max)
    for g in (W.rmat(14, 16, 2), W.bipartite_zipf(4096, 4096, 3), W.grid(40, 40, 47), W.rmat(12, 16, 45)):
        src, dst, cap = g.numpy()
        check_against_oracle(g.n, src, dst, cap, g.s, g.t, "bcsr", o)
    o.renumber = 1
    g = W.rmat(14, 16, 41)
    src, dst, cap = g.numpy()
    check_against_oracle(g.n, src, dst, cap, g.s, g.t, "bcsr", o)
