"""The batched and served workload at its stated sizes, against the oracle.

The stated stream is 4,096 instances of the seeded mix (workloads.batch_spec,
seeds 1000 + i): grids of side 32..512 with capacities U[1,255] and
unit-capacity bipartite graphs of 2^10..2^18 vertices per side.  This test
takes 512 of them: the first 448 of the stream plus its 32 largest grids
(up to 512 x 512) and its 32 largest bipartite graphs (up to 2^18 per side),
so the high-diameter grids and the largest matchings are included.  All of
them are solved in one batched launch and again through the
continuous-batching server with Poisson arrivals at the batched rate; every
value must equal the oracle's, and the served solves must overlap on the
device.
"""
import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_helpers import wb
from tests.oracle_pool import spec_values

pytestmark = pytest.mark.gpu


def _selection():
    specs = W.batch_spec(4096)
    grids = sorted((i for i, sp in enumerate(specs) if sp[0] == "grid"), key=lambda i: (-specs[i][1], i))[:32]
    bips = sorted((i for i, sp in enumerate(specs) if sp[0] == "bip"),
                  key=lambda i: (-specs[i][1], i))[:32]
    idx = sorted(set(range(448)) | set(grids) | set(bips))
    return [specs[i] for i in idx]


@pytest.mark.slow
def test_c5_mix_batched_and_served_equal_oracle():
    m = wb()
    from paper_2404_00270_gb300 import serve
    specs = _selection()
    assert max(sp[1] for sp in specs if sp[0] == "grid") == 512
    assert max(sp[1] for sp in specs if sp[0] == "bip") >= 250000
    refs = spec_values(specs)
    dev = torch.device("cuda:0")
    insts = [W.make_from_spec(sp, device=dev) for sp in specs]
    graphs = [m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, m.WBPR_BCSR) for g in insts]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    values = m.wbpr_maxflow_batch(graphs)
    ev1.record()
    torch.cuda.synchronize()
    assert values == refs
    rate = len(graphs) / (ev0.elapsed_time(ev1) / 1e3)
    for G in graphs:
        G.close()
    del graphs
    torch.cuda.empty_cache()
    rng = np.random.default_rng(11)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(insts)))
    reqs = [serve.Request(i, g.n, g.src, g.dst, g.cap, g.s, g.t, float(a))
            for i, (g, a) in enumerate(zip(insts, arrivals))]
    free_b, _ = torch.cuda.mem_get_info()
    out = serve.Server(int(0.5 * free_b)).run(reqs)
    assert [r.value for r in out] == refs
    summ = serve.latency_summary(out)
    assert summ["max_concurrent_on_device"] >= 2
    print(f"C5 mix, {len(insts)} instances: batched {rate:.0f} solves/s; served {summ['solves_per_s']:.0f} "
          f"solves/s, p50 {summ['p50_ms']:.0f} ms, p99 {summ['p99_ms']:.0f} ms, "
          f"up to {summ['max_concurrent_on_device']} solves at once on the device")


@pytest.mark.slow
def test_c5_full_stream_batched_equals_oracle():
    """All 4,096 instances of the stated stream in one batched launch."""
    m = wb()
    specs = W.batch_spec(4096)
    refs = spec_values(specs)
    dev = torch.device("cuda:0")
    graphs = []
    for sp in specs:
        g = W.make_from_spec(sp, device=dev)
        graphs.append(m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, m.WBPR_BCSR))
        del g
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    values = m.wbpr_maxflow_batch(graphs)
    ev1.record()
    torch.cuda.synchronize()
    for G in graphs:
        G.close()
    bad = [i for i, (a, b) in enumerate(zip(values, refs)) if a != b]
    assert not bad, bad[:10]
    print(f"C5 stream, 4096 instances in one batched launch: {ev0.elapsed_time(ev1):.0f} ms")


def test_batch_with_tuned_table_keeps_values():
    """Per-class tuned knobs (autotune.tune_batch) change no value."""
    m = wb()
    from paper_2404_00270_gb300 import autotune
    specs = W.batch_spec(48, base_seed=7000, grid_hi=96, bip_hi=1 << 13)
    refs = spec_values(specs)
    insts = [W.make_from_spec(sp, device="cuda:0") for sp in specs]
    table = autotune.tune_batch(insts, team=4, big_slots=1 << 13)
    assert table.entries
    graphs = [m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, m.WBPR_BCSR) for g in insts]
    autotune.apply_table(graphs, table)
    o = m.wbpr_get_options(graphs[0])
    o.batch_team, o.batch_big_slots = 4, 1 << 13
    m.wbpr_set_options(graphs[0], o)
    assert m.wbpr_maxflow_batch(graphs) == refs
    for G in graphs:
        G.close()
