"""Continuous-batching server for max-flow / matching requests.

Host-side scheduling only; every solve runs in the CUDA library through
``wbpr_maxflow_batch``.  Requests arrive over time (their graphs already
resident on the device as COO arrays).  The admission loop builds a request's
residual graph (``wbpr_build``) as soon as the device-memory footprint of the
requests in flight leaves room for it, and keeps it resident until its solve
returns.  Worker threads, each with its own CUDA stream and a slice of the
GPU (``grid_blocks``), repeatedly take every admitted request that is waiting
(up to ``max_batch``) and solve them together in one batched launch.  So
requests that arrive while others are on the GPU join the next batch of any
worker that frees up, and the batches of different workers overlap on the
device.  Latency is measured from a request's arrival to the return of its
batch.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import torch

from . import (WBPR_BCSR, wbpr_build, wbpr_default_options, wbpr_get_info, wbpr_maxflow_batch,
               load)


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

    @property
    def m(self) -> int:
        return int(self.src.numel())


def footprint_estimate(n: int, m: int) -> int:
    """Device bytes of a BCSR handle: 20 B per slot (at most 2 m slots),
    12 B per input arc, about 110 B per vertex of solver state."""
    return 40 * m + 12 * m + 110 * n


class Server:
    def __init__(self, memory_budget: int, workers: int = 2, max_batch: int = 512,
                 layout: int = WBPR_BCSR, device=None):
        load()
        self.device = torch.device(device or "cuda", torch.cuda.current_device())
        self.budget = int(memory_budget)
        self.workers = workers
        self.max_batch = max_batch
        self.layout = layout
        per_worker = 0
        props = torch.cuda.get_device_properties(self.device)
        # each worker's batches get an equal slice of the co-resident blocks
        per_worker = max(1, (props.multi_processor_count * 4) // workers)
        self.opts = wbpr_default_options()
        self.opts.grid_blocks = per_worker
        self._lock = threading.Condition()
        self._ready = collections.deque()
        self._in_use = 0
        self._stop = False
        self.batches = []

    # -- worker ---------------------------------------------------------------
    def _worker(self, t0: float):
        stream = torch.cuda.Stream(device=self.device)
        torch.cuda.set_device(self.device)
        while True:
            with self._lock:
                while not self._ready and not self._stop:
                    self._lock.wait(0.01)
                if not self._ready and self._stop:
                    return
                batch = []
                while self._ready and len(batch) < self.max_batch:
                    batch.append(self._ready.popleft())
            handles = [g for _, g in batch]
            values = wbpr_maxflow_batch(handles, stream)
            now = time.perf_counter() - t0
            for (req, g), v in zip(batch, values):
                req.value = v
                req.done = now
                g.close()
            with self._lock:
                for req, _ in batch:
                    self._in_use -= req.footprint
                self.batches.append((now, len(batch)))
                self._lock.notify_all()

    # -- admission loop ---------------------------------------------------------
    def run(self, requests):
        """Serve `requests` (sorted by arrival); returns them with results."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        arrived = collections.deque()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(t0,), daemon=True)
                   for _ in range(self.workers)]
        for th in threads:
            th.start()
        build_stream = torch.cuda.Stream(device=self.device)
        while pending or arrived:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                arrived.append(pending.popleft())
            admitted_any = False
            while arrived:
                req = arrived[0]
                need = footprint_estimate(req.n, req.m)
                with self._lock:
                    busy = self._in_use
                if busy > 0 and busy + need > self.budget:
                    break
                arrived.popleft()
                g = wbpr_build(req.n, req.m, req.src, req.dst, req.cap, req.s, req.t, self.layout,
                               self.opts, build_stream)
                req.footprint = max(need, wbpr_get_info(g)["device_bytes"])
                req.admitted = time.perf_counter() - t0
                with self._lock:
                    self._in_use += req.footprint
                    self._ready.append((req, g))
                    self._lock.notify_all()
                admitted_any = True
            if not admitted_any:
                with self._lock:
                    wait = 0.0005 if not pending else max(0.0, min(0.002, pending[0].arrival - now))
                    self._lock.wait(wait)
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        for th in threads:
            th.join()
        return requests


def latency_summary(requests) -> dict:
    lat = sorted(r.done - r.arrival for r in requests)
    n = len(lat)
    if n == 0:
        return {}
    first = min(r.arrival for r in requests)
    last = max(r.done for r in requests)
    q = lambda p: lat[min(n - 1, int(p * (n - 1) + 0.5))]
    return {"solves": n, "solves_per_s": n / max(1e-9, last - first), "p50_ms": 1e3 * q(0.50),
            "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * lat[-1], "makespan_s": last - first}
