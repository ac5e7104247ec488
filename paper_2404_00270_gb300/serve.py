"""Continuous-batching server for max-flow / matching requests.

Host-side admission only; every solve runs in the library's persistent
server kernel (``wbpr_server_start``).  Requests arrive over time with their
graphs already on the device as COO arrays.  The admission loop builds a
request's residual graph (``wbpr_build``) as soon as the device-memory
footprint of the requests in flight leaves room for it, and publishes it to
the kernel (``wbpr_server_submit``).  The kernel's first free team of the
request's size class starts solving it at once, while other requests are
still being solved.  The graph stays resident until its result is polled
(``wbpr_server_poll``), which frees its memory for the next admissions.
Latency is measured from a request's arrival to the poll that sees it done.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import torch

from . import (WBPR_BCSR, load, torch_allocator_enabled, use_torch_allocator, wbpr_build,
               wbpr_default_options, wbpr_get_info, wbpr_server_default_options,
               wbpr_server_poll, wbpr_server_start, wbpr_server_stop, wbpr_server_submit,
               wbpr_server_team_exits, wbpr_server_times)


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    src: torch.Tensor  # int32 on the device
    dst: torch.Tensor
    cap: torch.Tensor
    s: int
    t: int
    arrival: float      # seconds after the start of the run
    value: int | None = None
    admitted: float | None = None
    done: float | None = None
    footprint: int = 0
    build_ms: float = 0.0
    device_ns: tuple | None = None  # (start, end) of the solve on the device's globaltimer
    rejected: str | None = None     # why admission refused the request (it is not solved)

    @property
    def m(self) -> int:
        return int(self.src.numel())


def footprint_estimate(n: int, m: int) -> int:
    """Device bytes of a BCSR handle: 20 B per slot (at most 2 m slots),
    12 B per input arc, about 110 B per vertex of solver state."""
    return 40 * m + 12 * m + 110 * n


def admission(need: int, in_use: int, budget: int, busy: bool) -> str:
    """Admission decision for a request of footprint `need`: "reject" when it
    can never fit the budget, "wait" while the requests in flight (`busy`,
    holding `in_use` bytes) leave no room for it, else "admit"."""
    if need > budget:
        return "reject"
    if busy and in_use + need > budget:
        return "wait"
    return "admit"


class Server:
    """Admission by footprint in front of the persistent server kernel."""

    def __init__(self, memory_budget: int, layout: int = WBPR_BCSR, big_slots: int = 1 << 15,
                 team_blocks: int = 8, big_teams: int | None = None, small_blocks: int | None = None,
                 idle_ms: int = 60000, device=None, table=None):
        load()
        self.table = table   # autotune.Table: per-class options for each request's handle
        self.device = torch.device(device or "cuda", torch.cuda.current_device())
        self.budget = int(memory_budget)
        self.layout = layout
        self.opts = wbpr_server_default_options()
        self.opts.layout = layout
        self.opts.big_slots = big_slots
        # two server blocks per SM: the rest of every SM stays free for the
        # builds that admission runs while the server kernel is resident; they
        # are lean builds (wbpr_options.lean_build), whose largest blocks fit
        # in the registers two server blocks leave on an SM
        total = 2 * torch.cuda.get_device_properties(self.device).multi_processor_count
        if big_teams is None:
            big_teams = max(1, (total * 3 // 5) // team_blocks)
        if small_blocks is None:
            small_blocks = max(1, total - big_teams * team_blocks)
        self.opts.team_blocks = team_blocks
        self.opts.big_teams = big_teams
        self.opts.small_blocks = small_blocks
        self.opts.idle_ms = idle_ms
        self.build_opts = wbpr_default_options()
        self.build_opts.lean_build = 1
        self.in_use = 0
        self.peak_in_use = 0
        self.stall_s = 120.0

    def run(self, requests, max_inflight: int = 1 << 30):
        """Serve `requests` (sorted by arrival); returns them with results."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.opts.capacity = max(1, len(pending))
        arrived = collections.deque()
        outstanding = {}
        build_stream = torch.cuda.Stream(device=self.device)
        # While the persistent kernel runs, device allocations must be
        # stream-ordered (cudaMallocAsync, the library's own allocator): a
        # cudaMalloc from a caching allocator growing its pool would wait for
        # every stream, the server's included.
        restore_torch = torch_allocator_enabled()
        if restore_torch:
            use_torch_allocator(False)
        torch.cuda.synchronize()
        srv = wbpr_server_start(self.opts)
        t0 = time.perf_counter()
        last_progress = t0
        try:
            while pending or arrived or outstanding:
                now = time.perf_counter() - t0
                if time.perf_counter() - last_progress > self.stall_s:
                    raise RuntimeError(f"server made no progress for {self.stall_s} s")
                while pending and pending[0].arrival <= now:
                    arrived.append(pending.popleft())
                # admission: build and publish while the footprint fits
                while arrived and len(outstanding) < max_inflight:
                    req = arrived[0]
                    need = footprint_estimate(req.n, req.m)
                    decision = admission(need, self.in_use, self.budget, bool(outstanding))
                    if decision == "wait":
                        break
                    arrived.popleft()
                    if decision == "reject":
                        req.rejected = (f"footprint {need} B exceeds the memory budget of {self.budget} B")
                        req.done = time.perf_counter() - t0
                        last_progress = time.perf_counter()
                        continue
                    tb = time.perf_counter()
                    g = wbpr_build(req.n, req.m, req.src, req.dst, req.cap, req.s, req.t, self.layout,
                                   self.build_opts, build_stream)
                    req.build_ms = 1e3 * (time.perf_counter() - tb)
                    if self.table is not None:
                        from .autotune import apply_table
                        apply_table([g], self.table)
                    req.footprint = max(need, wbpr_get_info(g)["device_bytes"])
                    self.in_use += req.footprint
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    req.admitted = time.perf_counter() - t0
                    outstanding[wbpr_server_submit(srv, g)] = (req, g)
                # completions
                done = []
                for ticket, (req, g) in outstanding.items():
                    try:
                        v = wbpr_server_poll(srv, ticket)
                    except Exception as exc:
                        teams = self.opts.big_teams + self.opts.small_blocks
                        exits = wbpr_server_team_exits(srv, teams)
                        raise RuntimeError(
                            f"request {req.rid} (ticket class {ticket >> 40}, index {ticket & ((1 << 40) - 1)}) "
                            f"failed at t={time.perf_counter() - t0:.2f}s after admission at {req.admitted:.2f}s "
                            f"(build {req.build_ms:.1f} ms); "
                            f"team exit reasons {collections.Counter(exits)}") from exc
                    if v is not None:
                        req.value = v
                        req.done = time.perf_counter() - t0
                        req.device_ns = wbpr_server_times(srv, ticket)
                        done.append(ticket)
                if done or not outstanding:
                    last_progress = time.perf_counter()
                for ticket in done:
                    req, g = outstanding.pop(ticket)
                    g.close()
                    self.in_use -= req.footprint
                if not done and not arrived and pending:
                    time.sleep(max(0.0, min(0.0005, pending[0].arrival - (time.perf_counter() - t0))))
        finally:
            wbpr_server_stop(srv)
            for req, g in outstanding.values():
                g.close()
            if restore_torch:
                use_torch_allocator(True)
        return requests


def max_overlap(requests) -> int:
    """Most requests whose device solves were in progress at one instant."""
    ev = []
    for r in requests:
        if getattr(r, "device_ns", None):
            ev.append((r.device_ns[0], 1))
            ev.append((r.device_ns[1], -1))
    best = cur = 0
    for _, d in sorted(ev, key=lambda x: (x[0], x[1])):
        cur += d
        best = max(best, cur)
    return best


def latency_summary(requests) -> dict:
    requests = [r for r in requests if not getattr(r, "rejected", None)]
    lat = sorted(r.done - r.arrival for r in requests)
    n = len(lat)
    if n == 0:
        return {}
    first = min(r.arrival for r in requests)
    last = max(r.done for r in requests)
    q = lambda p: lat[min(n - 1, int(p * (n - 1) + 0.5))]
    return {"solves": n, "solves_per_s": n / max(1e-9, last - first), "p50_ms": 1e3 * q(0.50),
            "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * lat[-1], "makespan_s": last - first,
            "max_concurrent_on_device": max_overlap(requests)}
