"""Autotuner for the solver's speed knobs.

None of the knobs changes a result: the tile widths per degree class
(`small_tile`, `small_max_degree`, `warp_max_degree`), the vertices each
block covers (through `grid_blocks`), the global-relabel frequency
(`gr_ratio`) and the BFS direction rule (`bottom_up`).  The tuner times
phase-1 solves of one graph under a grid of candidates, checks that every
candidate finds the same flow value, and keeps the fastest.  Results are
stored in a JSON table keyed by a coarse graph class (size, mean degree and
hub skew), so later graphs of the same class start from the tuned options.
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import (Options, WBPR_BCSR, wbpr_build, wbpr_default_options, wbpr_get_info,
               wbpr_get_stats, wbpr_maxflow, wbpr_set_options)

KNOBS = ("small_tile", "small_max_degree", "warp_max_degree", "grid_blocks", "gr_ratio", "bottom_up")


def graph_class(n: int, slots: int, max_degree: int) -> str:
    """Coarse class of a graph: log2 of the vertex count, rounded mean
    degree bucket, and log2 of the hub skew (max degree / mean degree)."""
    mean = max(1.0, slots / max(1, n))
    return (f"n{int(math.log2(max(2, n)))}-d{int(math.log2(mean) + 0.5)}-"
            f"h{int(math.log2(max(1.0, max_degree / mean)) + 0.5)}")


def candidates(num_sms: int):
    tiles = [(4, 4), (8, 8), (16, 16)]
    warps = [256, 1024, 2048]
    grids = [0, num_sms, 2 * num_sms]
    ratios = [0.5, 1.0, 2.0]
    directions = [14, 0]
    for (tile, smax), wmax, grid, ratio, bu in itertools.product(tiles, warps, grids, ratios, directions):
        yield {"small_tile": tile, "small_max_degree": smax, "warp_max_degree": wmax,
               "grid_blocks": grid, "gr_ratio": ratio, "bottom_up": bu}


def _apply(opts: Options, cfg: dict) -> Options:
    for k, v in cfg.items():
        setattr(opts, k, v)
    return opts


def autotune(n, m, src, dst, cap, s, t, layout=WBPR_BCSR, reps: int = 2, limit: int | None = None,
             stream=None):
    """Returns (best config dict, best ms, [(config, ms), ...]).  Raises if two
    candidates disagree on the flow value (they cannot, unless something is
    broken)."""
    g = wbpr_build(n, m, src, dst, cap, s, t, layout, None, stream)
    try:
        info = wbpr_get_info(g)
        value = None
        trials = []
        for i, cfg in enumerate(candidates(info["num_sms"])):
            if limit is not None and i >= limit:
                break
            wbpr_set_options(g, _apply(wbpr_default_options(), cfg))
            best = math.inf
            for _ in range(reps):
                v = wbpr_maxflow(g, stream)
                if value is None:
                    value = v
                elif v != value:
                    raise RuntimeError(f"candidate {cfg} found flow {v}, another found {value}")
                best = min(best, wbpr_get_stats(g)["solve_ms"])
            trials.append((cfg, best))
        trials.sort(key=lambda x: x[1])
        return trials[0][0], trials[0][1], trials
    finally:
        g.close()


class Table:
    """Tuned options per graph class, kept in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def record(self, key: str, cfg: dict, ms: float):
        old = self.entries.get(key)
        if old is None or ms < old["ms"]:
            self.entries[key] = {"options": dict(cfg), "ms": ms}

    def options_for(self, n: int, slots: int, max_degree: int) -> Options:
        opts = wbpr_default_options()
        e = self.entries.get(graph_class(n, slots, max_degree))
        return _apply(opts, e["options"]) if e else opts

    def save(self, path: str | None = None):
        path = path or self.path
        with open(path, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
