"""Failure paths, made on the host or by device waits that run out, never by
a GPU fault.

* Allocation failure: an allocator hook (wbpr_set_allocator) that refuses
  the k-th request, for every k of a build: the build returns WBPR_ENOMEM
  and every block it did get is returned (no leak).
* Device wait limit: a grid barrier told to wait for one arrival more than
  the grid has (the test-only option barrier_extra) runs into
  barrier_timeout_ms; the solve returns WBPR_ETIMEOUT, and the same handle
  then solves correctly.
* Server idle limit: with no requests for idle_ms every team leaves the
  server kernel ("idle"), and a request submitted afterwards is reported as
  WBPR_ESTATE by the poll instead of being waited for.
* Serving admission: a request larger than the memory budget is rejected,
  the others are solved.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import wb

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT, ESTATE = -2, -4, -6


class _FailingAllocator:
    """Device allocations through torch's caching allocator, except that the
    request numbered `fail_at` (0-based) is refused.  Counts what is live."""

    def __init__(self, m, fail_at):
        self.m, self.fail_at = m, fail_at
        self.requests = 0
        self.live = {}
        A = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
        F = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
        self.cbs = (A(self._alloc), F(self._free))
        self.had_torch = m.torch_allocator_enabled()

    def _alloc(self, nbytes, stream, ctx):
        k = self.requests
        self.requests += 1
        if k == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        self.live[int(p)] = int(nbytes)
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        assert self.live.pop(int(ptr)) == int(nbytes)
        torch.cuda.caching_allocator_delete(int(ptr))

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


@pytest.mark.parametrize("layout", ["bcsr", "rcsr"])
def test_allocation_failure_at_every_point_of_a_build(layout):
    m = wb()
    L = m.WBPR_BCSR if layout == "bcsr" else m.WBPR_RCSR
    g = W.rmat(10, 8, 3)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
    o = m.wbpr_default_options()
    o.renumber = 1     # the renumbering's allocations too
    with _FailingAllocator(m, fail_at=-1) as probe:   # never fails: count the requests
        G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, L, o)
        assert m.wbpr_maxflow(G) == ref
        G.close()
    total = probe.requests
    assert total > 10 and not probe.live
    for k in range(total):
        with _FailingAllocator(m, fail_at=k) as hook:
            with pytest.raises(m.WbprError) as e:
                m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, L, o)
            assert e.value.status == ENOMEM, (k, e.value)
            torch.cuda.synchronize()
            assert not hook.live, (k, len(hook.live))   # every block it got was returned
    # the library still works afterwards
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, L, o)
    assert m.wbpr_maxflow(G) == ref
    G.close()


def test_barrier_wait_limit_reports_timeout_and_handle_survives():
    m = wb()
    g = W.grid(32, 32, 4)
    src, dst, cap = g.numpy()
    ref = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"]
    o = m.wbpr_default_options()
    o.barrier_extra = 1           # one arrival more than the grid has: the wait cannot end
    o.barrier_timeout_ms = 200
    o.grid_blocks = 8
    G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR, o)
    t0 = time.perf_counter()
    with pytest.raises(m.WbprError) as e:
        m.wbpr_maxflow(G)
    assert e.value.status == ETIMEOUT
    assert "wait point" in str(e.value)
    assert time.perf_counter() - t0 < 10.0
    o.barrier_extra = 0
    o.barrier_timeout_ms = 20000
    m.wbpr_set_options(G, o)
    assert m.wbpr_maxflow(G) == ref
    side = torch.empty(g.n, dtype=torch.uint8, device="cuda:0")
    assert m.wbpr_mincut(G, None, side) == ref
    G.close()


def test_server_idle_limit_then_poll_reports_state_error():
    m = wb()
    o = m.wbpr_server_default_options()
    o.big_teams, o.small_blocks, o.team_blocks, o.idle_ms = 0, 4, 1, 200
    srv = m.wbpr_server_start(o)
    try:
        t0 = time.perf_counter()
        exits = None
        while exits is None and time.perf_counter() - t0 < 30.0:
            time.sleep(0.05)
            exits = m.wbpr_server_team_exits(srv, 4)
        assert exits is not None, "the server kernel did not stop on its idle limit"
        assert list(exits) == [3, 3, 3, 3]          # every team left on the idle limit
        g = W.grid(8, 8, 1)
        src, dst, cap = g.numpy()
        G = m.wbpr_build(g.n, g.m, src, dst, cap, g.s, g.t, m.WBPR_BCSR)
        ticket = m.wbpr_server_submit(srv, G)
        with pytest.raises(m.WbprError) as e:
            m.wbpr_server_poll(srv, ticket)
        assert e.value.status == ESTATE
        G.close()
    finally:
        m.wbpr_server_stop(srv)


def test_serving_rejects_a_request_over_the_budget():
    m = wb()
    from paper_2404_00270_gb300 import serve
    dev = torch.device("cuda:0")
    insts = [W.grid(16, 16, 1), W.rmat(14, 16, 2), W.grid(12, 12, 2)]
    refs = []
    reqs = []
    for i, g in enumerate(insts):
        src, dst, cap = g.numpy()
        refs.append(oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t, False, False)["value"])
        d = g.to(dev)
        reqs.append(serve.Request(i, g.n, d.src, d.dst, d.cap, g.s, g.t, 0.001 * i))
    budget = 2 * max(serve.footprint_estimate(insts[k].n, insts[k].m) for k in (0, 2))
    assert serve.footprint_estimate(insts[1].n, insts[1].m) > budget
    out = serve.Server(budget, big_teams=1, team_blocks=4, small_blocks=8).run(reqs)
    assert out[1].rejected and out[1].value is None
    assert out[0].value == refs[0] and out[2].value == refs[2]
    assert not out[0].rejected and not out[2].rejected
    assert serve.latency_summary(out)["solves"] == 2
