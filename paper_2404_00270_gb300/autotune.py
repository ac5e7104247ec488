"""Autotuner for the solver's speed knobs.

None of the knobs changes a result: the tile widths per degree class
(`small_tile`, `small_max_degree`, `warp_max_degree`), the vertices each
block covers (through `grid_blocks`), the global-relabel frequency
(`gr_ratio`) and the BFS direction rule (`bottom_up`).  The tuner times
phase-1 solves of one graph under a grid of candidates, checks that every
candidate finds the same flow value, and keeps the fastest.  Results are
stored in a JSON table keyed by a coarse graph class (size, mean degree and
hub skew), so later graphs of the same class start from the tuned options.

For batches (wbpr_maxflow_batch and the server) tune_batch() times each
class's largest instance the way the batch solves it (one block, or a team
of blocks for large instances) and apply_table() sets every handle of a
batch to its class's entry before the batched launch.
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import (Options, WBPR_BCSR, wbpr_build, wbpr_default_options, wbpr_get_info, wbpr_get_options,
               wbpr_get_stats, wbpr_maxflow, wbpr_set_options)

KNOBS = ("small_tile", "small_max_degree", "warp_max_degree", "grid_blocks", "gr_ratio", "bottom_up")
# bottom_up_edges (the form of the direction rule) is left at its default.


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


def batch_candidates():
    """Knobs a batched solve can vary per instance (the server kernel's tile
    width is fixed at 8 lanes, and the team size is the batch's)."""
    for wmax, ratio, bu in itertools.product([256, 1024], [0.5, 1.0, 2.0, 4.0], [14, 0]):
        yield {"warp_max_degree": wmax, "gr_ratio": ratio, "bottom_up": bu}


def tune_batch(instances, layout=WBPR_BCSR, team: int = 16, big_slots: int = 1 << 15, reps: int = 1,
               stream=None, table: "Table | None" = None):
    """Tunes the batch knobs per graph class.  For every class among
    `instances` (objects with n, m, src, dst, cap, s, t), its largest
    instance is solved as a batch solves it -- on a grid of one block, or of
    `team` blocks when it has more than `big_slots` residual slots -- under
    every batch candidate; the fastest is recorded.  Returns the table."""
    table = table or Table()
    reps_by_class = {}
    for inst in instances:
        g = wbpr_build(inst.n, inst.m, inst.src, inst.dst, inst.cap, inst.s, inst.t, layout, None, stream)
        info = wbpr_get_info(g)
        g.close()
        key = graph_class(info["n"], info["slots"], info["max_degree"])
        if key not in reps_by_class or info["slots"] > reps_by_class[key][1]:
            reps_by_class[key] = (inst, info["slots"])
    for key, (inst, slots) in sorted(reps_by_class.items()):
        blocks = team if slots > big_slots else 1
        g = wbpr_build(inst.n, inst.m, inst.src, inst.dst, inst.cap, inst.s, inst.t, layout, None, stream)
        try:
            value = None
            for cfg in batch_candidates():
                o = _apply(wbpr_default_options(), cfg)
                o.grid_blocks = blocks
                wbpr_set_options(g, o)
                best = math.inf
                for _ in range(reps):
                    v = wbpr_maxflow(g, stream)
                    if value is None:
                        value = v
                    elif v != value:
                        raise RuntimeError(f"candidate {cfg} found flow {v}, another found {value}")
                    best = min(best, wbpr_get_stats(g)["solve_ms"])
                table.record(key, cfg, best)
        finally:
            g.close()
    return table


def apply_table(graphs, table: "Table"):
    """Sets every handle's options to its class's tuned knobs (unknown
    classes keep theirs)."""
    for g in graphs:
        info = wbpr_get_info(g)
        e = table.entries.get(graph_class(info["n"], info["slots"], info["max_degree"]))
        if e:
            wbpr_set_options(g, _apply(wbpr_get_options(g), e["options"]))


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
