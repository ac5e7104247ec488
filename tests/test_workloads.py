"""The seeded input generators: counter-based SplitMix64 and graph shapes."""
import numpy as np
import torch

import workloads as W


def test_mix64_matches_integer_definition():
    zs = [0, 1, 2, 12345, (1 << 63) - 1, 1 << 63, (1 << 64) - 1, 0x9E3779B97F4A7C15]
    t = torch.tensor([W._s64(z) for z in zs], dtype=torch.int64)
    got = [x & W.MASK64 for x in W._mix64(t).tolist()]
    assert got == [W.mix64_reference(z) for z in zs]
    # SplitMix64 with seed 0: first output is mix64(0x9E3779B97F4A7C15).
    assert W.mix64_reference(W.GAMMA) == 0xE220A8397B1DCDAF


def test_draws_are_deterministic_and_in_range():
    c = torch.arange(100000, dtype=torch.int64)
    a = W.draw_int(7, 3, c, 1, 100)
    b = W.draw_int(7, 3, c, 1, 100)
    assert torch.equal(a, b)
    assert int(a.min()) == 1 and int(a.max()) == 100
    assert abs(float(a.float().mean()) - 50.5) < 0.5
    assert not torch.equal(a, W.draw_int(8, 3, c, 1, 100))


def test_grid_shape():
    g = W.grid(64, 64, 1)
    assert g.n == 4098 and g.m == 16256 and g.s == 4096 and g.t == 4097
    src, dst, cap = g.numpy()
    assert cap[:16128].min() >= 1 and cap[:16128].max() <= 100
    assert (cap[16128:] == 1000).all()
    # every grid arc joins 4-neighbours
    r1, c1, r2, c2 = src[:16128] // 64, src[:16128] % 64, dst[:16128] // 64, dst[:16128] % 64
    assert (np.abs(r1 - r2) + np.abs(c1 - c2) == 1).all()


def test_rmat_small_properties():
    g = W.rmat(12, 16, 3)
    src, dst, cap = g.numpy()
    assert (src != dst).all()
    key = src.astype(np.int64) * g.n + dst
    assert np.unique(key).size == key.size
    assert (np.diff(key) > 0).all()
    assert cap.min() >= 1 and cap.max() <= 1000
    outdeg = np.bincount(src, minlength=g.n)
    assert outdeg[g.s] == outdeg.max()


def test_zipf_degree_law_mean():
    thr = W.zipf_degree_thresholds(2.1, 0.9213, 4096)
    p = np.diff(np.concatenate([[0], thr])).astype(np.float64) / float(1 << 53)
    mean = float((p * np.arange(1, 4097)).sum())
    assert abs(mean - 8.0) < 0.01


def test_bipartite_shape():
    g = W.bipartite_zipf(1 << 10, 1 << 10, 3)
    src, dst, cap = g.numpy()
    nl = 1 << 10
    lr = g.meta["lr_edges"]
    assert g.meta["max_left_degree"] == 4096
    assert (src[:lr] < nl).all() and (dst[:lr] >= nl).all()
    assert (cap == 1).all() and g.m == lr + 2 * nl


def test_vision_grid_shape_and_closed_form():
    """A uniform image (no noise, one block) cuts every pixel alone at
    min(I, 255 - I) = 65, whichever intensity the block drew: no smoothness
    arc is cut, since all pixels take the same side."""
    import oracle
    oracle.build()
    for seed in (1, 2, 3):
        g = W.vision_grid(16, 20, seed, block=32, noise=0)
        assert g.n == 16 * 20 + 2 and (g.s, g.t) == (320, 321)
        grid_arcs = 4 * 16 * 20 - 2 * 16 - 2 * 20
        assert g.m == grid_arcs + 2 * 320
        src, dst, cap = g.numpy()
        assert ((src[grid_arcs:grid_arcs + 320] == 320) & (dst[grid_arcs + 320:] == 321)).all()
        assert set(cap[grid_arcs:grid_arcs + 320].tolist()) <= {65, 190}
        assert (cap[grid_arcs:grid_arcs + 320] + cap[grid_arcs + 320:] == 255).all()
        r = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)
        assert r["value"] == 65 * 320
    g = W.vision_grid(48, 40, 5, block=16)
    src, dst, cap = g.numpy()
    assert oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"] == \
        oracle.maxflow_dinic(g.n, src, dst, cap, g.s, g.t)["value"]
