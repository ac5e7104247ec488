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
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import wb

pytestmark = pytest.mark.gpu


def _bcsr_on_device(m, G, dev):
    off = torch.from_numpy(m.wbpr_export(G, "offsets")).to(dev)
    col = torch.from_numpy(m.wbpr_export(G, "col")).to(dev)
    cap = torch.from_numpy(m.wbpr_export(G, "cap")).to(dev)
    rev = torch.from_numpy(m.wbpr_export(G, "rev").view(np.int32)).to(dev)
    return off, col, cap, rev


def _input_ids(m):
    o = m.wbpr_default_options()
    o.renumber = 0     # exported arrays in input ids, so s and t carry over
    return o


def _instances():
    yield W.grid(64, 64, 1)
    yield W.rmat(12, 16, 7)
    yield W.bipartite_zipf(1 << 10, 1 << 10, 5)


class _CountingAllocator:
    """An allocator hook (wbpr_set_allocator) that refuses and counts every
    request, installed only around the allocation-free calls."""

    def __init__(self, m):
        self.m = m
        self.calls = 0
        self.had_torch = m.torch_allocator_enabled()
        A = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
        F = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
        self.cbs = (A(self._alloc), F(self._free))

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        return None

    def _free(self, ptr, nbytes, stream, ctx):
        self.calls += 1

    def __enter__(self):
        lib = self.m.load()
        assert lib.wbpr_set_allocator(ctypes.cast(self.cbs[0], ctypes.c_void_p),
                                      ctypes.cast(self.cbs[1], ctypes.c_void_p), None) == 0
        return self

    def __exit__(self, *exc):
        if self.had_torch:
            self.m.use_torch_allocator(True)
        else:
            self.m.load().wbpr_set_allocator(None, None, None)


def test_noalloc_matches_maxflow_twice_in_a_row():
    m = wb()
    dev = torch.device("cuda:0")
    for inst in _instances():
        src, dst, cap = inst.numpy()
        G = m.wbpr_build(inst.n, inst.m, src, dst, cap, inst.s, inst.t, m.WBPR_BCSR, _input_ids(m))
        expected = m.wbpr_maxflow(G)
        assert expected == oracle.maxflow_pr(inst.n, src, dst, cap, inst.s, inst.t, False, False)["value"]
        off, col, capd, rev = _bcsr_on_device(m, G, dev)
        slots = col.numel()
        assert inst.n <= m.NOALLOC_MAX_VERTICES and slots <= m.NOALLOC_MAX_SLOTS
        for call in range(2):
            value = torch.full((1,), -1, dtype=torch.int64, device=dev)
            residual = torch.full((slots,), -1, dtype=torch.int32, device=dev)
            torch.cuda.synchronize()
            free_before, _ = torch.cuda.mem_get_info()
            with _CountingAllocator(m) as hook:
                m.wbpr_maxflow_bcsr_noalloc(inst.n, slots, inst.s, inst.t, off, col, capd, rev, None,
                                            value, residual)
            free_after, _ = torch.cuda.mem_get_info()
            assert hook.calls == 0, (inst.name, call)
            if call == 1:   # the first call may load the library's device code
                assert free_after == free_before, (inst.name, free_before - free_after)
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


def test_noalloc_rejects_malformed_arrays():
    """Arrays that break the BCSR invariants are refused before any solve."""
    m = wb()
    dev = torch.device("cuda:0")
    g = W.grid(16, 16, 3)
    src, dst, cap = g.numpy()
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR, _input_ids(m))
    off, col, capd, rev = _bcsr_on_device(m, G, dev)
    G.close()
    slots = col.numel()
    value = torch.zeros(1, dtype=torch.int64, device=dev)
    bad_off = off.clone()
    bad_off[-1] = slots - 1                      # off[n] != slots
    bad_col = col.clone()
    bad_col[3] = g.n                             # neighbour id out of range
    bad_rev = rev.clone()
    bad_rev[[0, 1]] = bad_rev[[1, 0]]            # pairing broken
    bad_cap = capd.clone()
    bad_cap[5] = -1                              # negative capacity
    for args in ((bad_off, col, capd, rev), (off, bad_col, capd, rev), (off, col, capd, bad_rev),
                 (off, col, bad_cap, rev)):
        with pytest.raises(m.WbprError) as e:
            m.wbpr_maxflow_bcsr_noalloc(g.n, slots, g.s, g.t, *args, None, value)
        assert e.value.status == -1
    # the well-formed arrays still solve afterwards
    m.wbpr_maxflow_bcsr_noalloc(g.n, slots, g.s, g.t, off, col, capd, rev, None, value)
    assert int(value.item()) == oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
