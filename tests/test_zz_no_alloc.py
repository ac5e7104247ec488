"""The allocation-free entry point, wbpr_maxflow_bcsr_noalloc.

Some callers of this library may not allocate device memory while they run:
code inside a framework's execution phase that forbids allocation, real-time
loops with a device memory budget fixed in advance, or embedders without a
CUDA allocator of their own.  For them the library solves small BCSR graphs
out of one fixed device array instead of allocating.  These tests call that
entry point through the C ABI, twice in a row (the array keeps the previous
call's contents, so the second call checks that the call clears what it
must), and compare it with the ordinary wbpr_maxflow on the same graph:
flow values are exact integers, so they must be equal.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_helpers import wb

pytestmark = pytest.mark.gpu


def _bcsr_on_device(m, G, dev):
    off = torch.from_numpy(m.wbpr_export(G, "offsets")).to(dev)
    col = torch.from_numpy(m.wbpr_export(G, "col")).to(dev)
    cap = torch.from_numpy(m.wbpr_export(G, "cap")).to(dev)
    rev = torch.from_numpy(m.wbpr_export(G, "rev").view(np.int32)).to(dev)
    return off, col, cap, rev


def _instances():
    yield W.grid(64, 64, 1)
    yield W.rmat(12, 16, 7)
    yield W.bipartite_zipf(1 << 10, 1 << 10, 5)


def test_noalloc_matches_maxflow_twice_in_a_row():
    m = wb()
    dev = torch.device("cuda:0")
    for inst in _instances():
        src, dst, cap = inst.numpy()
        G = m.wbpr_build(inst.n, inst.m, src, dst, cap, inst.s, inst.t, m.WBPR_BCSR)
        expected = m.wbpr_maxflow(G)
        off, col, capd, rev = _bcsr_on_device(m, G, dev)
        slots = col.numel()
        assert inst.n <= m.NOALLOC_MAX_VERTICES and slots <= m.NOALLOC_MAX_SLOTS
        for call in range(2):
            value = torch.full((1,), -1, dtype=torch.int64, device=dev)
            residual = torch.full((slots,), -1, dtype=torch.int32, device=dev)
            m.wbpr_maxflow_bcsr_noalloc(inst.n, slots, inst.s, inst.t, off, col, capd, rev, None,
                                        value, residual)
            assert int(value.item()) == expected, (inst.name, call)
            # the residual capacities of each merged pair still add up to the
            # pair's total capacity, and none is negative
            r = residual.cpu().numpy().astype(np.int64)
            c = capd.cpu().numpy().astype(np.int64)
            rv = rev.cpu().numpy().view(np.uint32).astype(np.int64)
            assert (r >= 0).all()
            assert np.array_equal(r + r[rv], c + c[rv])
        G.close()


def test_noalloc_rejects_graphs_beyond_its_fixed_size():
    m = wb()
    dev = torch.device("cuda:0")
    off = torch.zeros(3, dtype=torch.int64, device=dev)
    value = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(m.WbprError) as e:
        m.wbpr_maxflow_bcsr_noalloc(m.NOALLOC_MAX_VERTICES + 1, 0, 0, 1, off, None, None, None,
                                    None, value)
    assert e.value.status == -1
    z32 = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(m.WbprError) as e:
        m.wbpr_maxflow_bcsr_noalloc(2, m.NOALLOC_MAX_SLOTS + 1, 0, 1, off, z32, z32, z32, None, value)
    assert e.value.status == -1
