"""Seeded synthetic max-flow inputs.

This module only draws inputs: it holds none of the max-flow arithmetic, and
both the CUDA path and the CPU oracle take their graphs from it.  Every
generator returns a :class:`FlowInstance` (n, int32 arc arrays src/dst/cap,
source s, sink t) on the requested torch device.  Results do not depend on
the device: random numbers come from a counter-based SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014:
output k of the stream started at state x is mix64(x + k * 0x9E3779B97F4A7C15))
evaluated in wrapping 64-bit integer arithmetic, and every table that needs
floating point is computed on the host in float64 and turned into integer
thresholds before it reaches the device.

The shapes follow the workloads the paper measures on (power-law SNAP
graphs and DIMACS generators for max-flow, KONECT bipartite graphs for
matching); the real datasets are not used.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """A 64-bit pattern as the signed value torch.int64 stores."""
    x &= MASK64
    return x - (1 << 64) if x >> 63 else x


def _mix64_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    return z ^ _lsr(z, 31)


def stream_start(seed: int, stream: int) -> int:
    """Start state of stream `stream` of seed `seed` (a SplitMix64 output)."""
    return _mix64_int((seed & MASK64) * GAMMA + (stream & MASK64) * 0xD1B54A32D192ED03)


def draw64(seed: int, stream: int, counter: torch.Tensor) -> torch.Tensor:
    """64-bit random bit patterns, one per counter value (int64 tensor)."""
    x0 = _s64(stream_start(seed, stream))
    return _mix64(counter * _s64(GAMMA) + x0)


def draw_u32(seed: int, stream: int, counter: torch.Tensor) -> torch.Tensor:
    """Uniform integers in [0, 2^32) as int64."""
    return _lsr(draw64(seed, stream, counter), 32)


def draw_int(seed: int, stream: int, counter: torch.Tensor, lo: int, hi: int) -> torch.Tensor:
    """Uniform integers in [lo, hi] (multiply-shift of a 32-bit draw)."""
    span = hi - lo + 1
    assert 0 < span <= (1 << 31)
    return lo + ((draw_u32(seed, stream, counter) * span) >> 32)


def mix64_reference(z: int) -> int:
    """Python-integer SplitMix64 finaliser (used by tests of the tensor form)."""
    return _mix64_int(z)


@dataclasses.dataclass
class FlowInstance:
    name: str
    n: int
    src: torch.Tensor   # int32 [m]
    dst: torch.Tensor   # int32 [m]
    cap: torch.Tensor   # int32 [m]
    s: int
    t: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.numel())

    def to(self, device) -> "FlowInstance":
        return dataclasses.replace(self, src=self.src.to(device), dst=self.dst.to(device),
                                   cap=self.cap.to(device))

    def numpy(self):
        return (self.src.cpu().numpy(), self.dst.cpu().numpy(), self.cap.cpu().numpy())


# --------------------------------------------------------------------------
# 2-D 4-connected grid (the vision-style max-flow network; DIMACS-like).
# Vertex id = row * cols + col; s = rows*cols, t = rows*cols + 1.
# Arcs in row-major vertex order, per vertex: right, left, down, up (those
# that exist), each with its own capacity; then s -> (r, 0) and
# (r, cols-1) -> t for r = 0..rows-1 with capacity `term_cap`.
# --------------------------------------------------------------------------
def grid(rows: int, cols: int, seed: int, cap_lo: int = 1, cap_hi: int = 100,
         term_cap: int = 1000, uniform_cap: int | None = None, device="cpu") -> FlowInstance:
    dev = torch.device(device)
    r = torch.arange(rows, device=dev, dtype=torch.int64).repeat_interleave(cols)
    c = torch.arange(cols, device=dev, dtype=torch.int64).repeat(rows)
    v = r * cols + c
    dirs = [(0, 1), (0, -1), (1, 0), (-1, 0)]   # right, left, down, up
    srcs, dsts, oks = [], [], []
    for dr, dc in dirs:
        rr, cc = r + dr, c + dc
        ok = (rr >= 0) & (rr < rows) & (cc >= 0) & (cc < cols)
        srcs.append(v)
        dsts.append(rr * cols + cc)
        oks.append(ok)
    src = torch.stack(srcs, 1).reshape(-1)
    dst = torch.stack(dsts, 1).reshape(-1)
    ok = torch.stack(oks, 1).reshape(-1)
    src, dst = src[ok], dst[ok]
    k = src.numel()
    if uniform_cap is not None:
        cap = torch.full((k,), int(uniform_cap), dtype=torch.int64, device=dev)
    else:
        cap = draw_int(seed, 200, torch.arange(k, device=dev, dtype=torch.int64), cap_lo, cap_hi)
    nv = rows * cols
    s, t = nv, nv + 1
    rows_t = torch.arange(rows, device=dev, dtype=torch.int64)
    src = torch.cat([src, torch.full((rows,), s, device=dev, dtype=torch.int64),
                     rows_t * cols + (cols - 1)])
    dst = torch.cat([dst, rows_t * cols, torch.full((rows,), t, device=dev, dtype=torch.int64)])
    cap = torch.cat([cap, torch.full((2 * rows,), term_cap, device=dev, dtype=torch.int64)])
    return FlowInstance(f"grid{rows}x{cols}", nv + 2, src.int(), dst.int(), cap.int(), s, t,
                        {"rows": rows, "cols": cols, "seed": seed})


# --------------------------------------------------------------------------
# Vision-style segmentation network (the image-segmentation use of minimum
# cuts the paper's §1 cites): an R x C image, pixel p = row * C + col,
# s = R*C, t = R*C + 1.  Every pixel has a source arc s -> p with the
# foreground term and a sink arc p -> t with the background term, and each of
# its 4 neighbours q an arc p -> q with a smoothness capacity.  The image is a
# seeded synthetic intensity field in integer arithmetic only: a
# checkerboard of blocks of side `block` (bright or dark by a draw per
# block), plus uniform noise in [-noise, noise], clamped to [0, 255].
#   s -> p: I(p);  p -> t: 255 - I(p);  p -> q: max(1, lam - |I(p) - I(q)| / 4)
# Arcs come in row-major pixel order, per pixel: right, left, down, up (those
# that exist), then every s -> p, then every p -> t.
# --------------------------------------------------------------------------
def vision_grid(rows: int, cols: int, seed: int, block: int = 64, noise: int = 60, lam: int = 48,
                device="cpu") -> FlowInstance:
    dev = torch.device(device)
    nv = rows * cols
    pix = torch.arange(nv, device=dev, dtype=torch.int64)
    r, c = pix // cols, pix % cols
    nbc = (cols + block - 1) // block
    blk = (r // block) * nbc + (c // block)
    bright = draw_int(seed, 700, blk, 0, 1)
    base = torch.where(bright == 1, torch.full_like(blk, 190), torch.full_like(blk, 65))
    img = (base + draw_int(seed, 701, pix, -noise, noise)).clamp(0, 255)
    dirs = [(0, 1), (0, -1), (1, 0), (-1, 0)]   # right, left, down, up
    srcs, dsts, oks = [], [], []
    for dr, dc in dirs:
        rr, cc = r + dr, c + dc
        ok = (rr >= 0) & (rr < rows) & (cc >= 0) & (cc < cols)
        srcs.append(pix)
        dsts.append((rr * cols + cc).clamp(0, nv - 1))
        oks.append(ok)
    src = torch.stack(srcs, 1).reshape(-1)
    dst = torch.stack(dsts, 1).reshape(-1)
    ok = torch.stack(oks, 1).reshape(-1)
    src, dst = src[ok], dst[ok]
    smooth = torch.clamp(lam - (img[src] - img[dst]).abs() // 4, min=1)
    s, t = nv, nv + 1
    src = torch.cat([src, torch.full((nv,), s, device=dev, dtype=torch.int64), pix])
    dst = torch.cat([dst, pix, torch.full((nv,), t, device=dev, dtype=torch.int64)])
    cap = torch.cat([smooth, img, 255 - img])
    return FlowInstance(f"vision{rows}x{cols}", nv + 2, src.int(), dst.int(), cap.int(), s, t,
                        {"rows": rows, "cols": cols, "seed": seed, "block": block, "noise": noise, "lam": lam})


# --------------------------------------------------------------------------
# R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each of edge_factor * 2^scale
# edges picks, at each of `scale` levels, one quadrant with probabilities
# (a, b, c, d); quadrant b sets the destination bit, c the source bit, d both.
# Self-loops and duplicate (src, dst) pairs are removed; arcs come out sorted
# by (src, dst).  Capacities are drawn from the arc's (src, dst) key, so they
# do not depend on the order of generation.  s = the vertex of largest
# out-degree, t = the vertex of largest in-degree other than s (lowest id on
# ties).
# --------------------------------------------------------------------------
def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
         cap_lo: int = 1, cap_hi: int = 1000, device="cpu", chunk: int = 1 << 26) -> FlowInstance:
    dev = torch.device(device)
    n = 1 << scale
    M = edge_factor << scale
    ta = int(round(a * 2 ** 32))
    tab = int(round((a + b) * 2 ** 32))
    tabc = int(round((a + b + c) * 2 ** 32))
    keys = []
    for lo in range(0, M, chunk):
        idx = torch.arange(lo, min(M, lo + chunk), device=dev, dtype=torch.int64)
        src = torch.zeros_like(idx)
        dst = torch.zeros_like(idx)
        for level in range(scale):
            r = draw_u32(seed, 1 + level, idx)
            sbit = (r >= tab).long()
            dbit = (((r >= ta) & (r < tab)) | (r >= tabc)).long()
            src = src * 2 + sbit
            dst = dst * 2 + dbit
            del r, sbit, dbit
        keep = src != dst
        keys.append(((src << scale) | dst)[keep])
        del idx, src, dst, keep
    key = torch.unique(torch.cat(keys))
    del keys
    src = (key >> scale).int()
    dst = (key & (n - 1)).int()
    cap = draw_int(seed, 100, key, cap_lo, cap_hi).int()
    del key
    outdeg = torch.bincount(src.long(), minlength=n)
    indeg = torch.bincount(dst.long(), minlength=n)
    s = int(torch.argmax(outdeg).item())
    indeg[s] = -1
    t = int(torch.argmax(indeg).item())
    return FlowInstance(f"rmat{scale}", n, src, dst, cap, s, t,
                        {"scale": scale, "edge_factor": edge_factor, "seed": seed,
                         "max_out": int(outdeg.max().item()), "max_in": int(indeg.max().item())})


# --------------------------------------------------------------------------
# Multi-source / multi-sink instances (the construction of §4.1): k source /
# sink pairs on one graph, joined by a super source S* = n (arcs S* -> s_i)
# and a super sink T* = n + 1 (arcs t_i -> T*), appended after the graph's
# arcs in pair order.  Each super arc carries the total capacity of the arcs
# leaving s_i (resp. entering t_i), capped at 2^31 - 1, so it never limits
# the flow.
# --------------------------------------------------------------------------
def multi_terminal(inst: FlowInstance, sources, sinks, name: str | None = None) -> FlowInstance:
    sources = [int(x) for x in sources]
    sinks = [int(x) for x in sinks]
    if not sources or len(set(sources)) != len(sources) or len(set(sinks)) != len(sinks) or \
            set(sources) & set(sinks):
        raise ValueError("need distinct sources and sinks, disjoint from each other")
    src, dst, cap = (x.cpu().long() for x in (inst.src, inst.dst, inst.cap))
    n = inst.n
    out_cap = torch.zeros(n, dtype=torch.int64).index_add_(0, src, cap)
    in_cap = torch.zeros(n, dtype=torch.int64).index_add_(0, dst, cap)
    S, T = n, n + 1
    big = (1 << 31) - 1
    s_idx = torch.tensor(sources, dtype=torch.int64)
    t_idx = torch.tensor(sinks, dtype=torch.int64)
    src2 = torch.cat([src, torch.full_like(s_idx, S), t_idx])
    dst2 = torch.cat([dst, s_idx, torch.full_like(t_idx, T)])
    cap2 = torch.cat([cap, out_cap[s_idx].clamp(max=big), in_cap[t_idx].clamp(max=big)])
    dev = inst.src.device
    return FlowInstance(name or f"{inst.name}-multi{len(sources)}", n + 2, src2.int().to(dev), dst2.int().to(dev),
                        cap2.int().to(dev), S, T, dict(inst.meta, sources=sources, sinks=sinks))


def far_pairs(inst: FlowInstance, k: int):
    """k source / sink pairs far apart: the k largest out-degree vertices
    (lowest id on ties) are the sources; each takes as sink the vertex
    farthest from it by BFS over the arcs (lowest id on ties) among those it
    reaches that are neither a source nor an earlier sink.  A source that
    reaches no such vertex is skipped."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    src, dst, _ = inst.numpy()
    n = inst.n
    outdeg = np.bincount(src, minlength=n)
    order = np.lexsort((np.arange(n), -outdeg))
    cand = [int(v) for v in order[: 4 * k] if outdeg[v] > 0]
    A = sp.csr_matrix((np.ones(src.size), (src, dst)), shape=(n, n))
    sources, sinks = [], []
    for s0 in cand:
        if len(sources) == k:
            break
        if s0 in sinks:
            continue
        d = shortest_path(A, unweighted=True, directed=True, indices=[s0])[0]
        taken = set(cand[: 4 * k]) | set(sinks) | {s0}
        best, far = -1, -1.0
        for v in np.flatnonzero(np.isfinite(d)):
            v = int(v)
            if v in taken:
                continue
            if d[v] > far:
                best, far = v, d[v]
        if best >= 0:
            sources.append(s0)
            sinks.append(best)
    return sources, sinks


def rmat_multi(scale: int, edge_factor: int, seed: int, k: int, device="cpu") -> FlowInstance:
    """R-MAT graph (as :func:`rmat`) with k far-apart source / sink pairs
    joined by a super source and a super sink."""
    base = rmat(scale, edge_factor, seed)
    sources, sinks = far_pairs(base, k)
    return multi_terminal(base, sources, sinks, f"rmat{scale}-multi{len(sources)}").to(device)


# --------------------------------------------------------------------------
# Bipartite matching as unit-capacity max-flow.  Left vertices 0..nl-1,
# right vertices nl..nl+nr-1, s = nl+nr, t = nl+nr+1.  Left degrees follow a
# discrete Zipf-Mandelbrot law p(d) ~ (d + delta)^(-exponent) on [1, dmax]
# (delta = 0.9213 makes the mean 8 for exponent 2.1, dmax 4096); left vertex
# 0 has degree dmax.  Each left vertex picks uniform right endpoints;
# duplicate (left, right) pairs are dropped.  Arcs: L->R sorted by (left,
# right), then s->L for every left vertex, then R->t for every right vertex,
# all capacity 1.
# --------------------------------------------------------------------------
def zipf_degree_thresholds(exponent: float, delta: float, dmax: int) -> np.ndarray:
    d = np.arange(1, dmax + 1, dtype=np.float64)
    p = (d + delta) ** (-exponent)
    cdf = np.cumsum(p) / p.sum()
    thr = np.floor(cdf * float(1 << 53)).astype(np.int64)
    thr[-1] = 1 << 53
    return thr


def bipartite_zipf(nl: int, nr: int, seed: int, exponent=2.1, delta=0.9213, dmax=4096,
                   device="cpu") -> FlowInstance:
    dev = torch.device(device)
    thr = torch.from_numpy(zipf_degree_thresholds(exponent, delta, dmax)).to(dev)
    u = torch.arange(nl, device=dev, dtype=torch.int64)
    x = _lsr(draw64(seed, 300, u), 11)                    # uniform in [0, 2^53)
    deg = torch.searchsorted(thr, x, right=True) + 1
    deg = torch.clamp(deg, max=dmax)
    deg[0] = dmax
    total = int(deg.sum().item())
    left = torch.repeat_interleave(u, deg)
    pos = torch.arange(total, device=dev, dtype=torch.int64)
    right = draw_int(seed, 301, pos, 0, nr - 1)
    key = torch.unique(left * nr + right)
    left = key // nr
    right = key % nr
    s, t = nl + nr, nl + nr + 1
    src = torch.cat([left, torch.full((nl,), s, device=dev, dtype=torch.int64),
                     torch.arange(nl, nl + nr, device=dev, dtype=torch.int64)])
    dst = torch.cat([nl + right, torch.arange(nl, device=dev, dtype=torch.int64),
                     torch.full((nr,), t, device=dev, dtype=torch.int64)])
    cap = torch.ones(src.numel(), device=dev, dtype=torch.int32)
    return FlowInstance(f"bipartite{nl}x{nr}", nl + nr + 2, src.int(), dst.int(), cap, s, t,
                        {"nl": nl, "nr": nr, "seed": seed, "lr_edges": int(key.numel()),
                         "max_left_degree": int(deg.max().item())})


# --------------------------------------------------------------------------
# Uniform bipartite instance with Poisson left degrees (batch mix).
# --------------------------------------------------------------------------
def _poisson_thresholds(mean: float, kmax: int) -> np.ndarray:
    k = np.arange(0, kmax + 1, dtype=np.float64)
    logp = -mean + k * math.log(mean) - np.array([math.lgamma(x + 1) for x in k])
    cdf = np.cumsum(np.exp(logp))
    cdf /= cdf[-1]
    thr = np.floor(cdf * float(1 << 53)).astype(np.int64)
    thr[-1] = 1 << 53
    return thr


def bipartite_poisson(nl: int, nr: int, mean_degree: int, seed: int, device="cpu") -> FlowInstance:
    dev = torch.device(device)
    kmax = max(4 * mean_degree + 40, 64)
    thr = torch.from_numpy(_poisson_thresholds(float(mean_degree), kmax)).to(dev)
    u = torch.arange(nl, device=dev, dtype=torch.int64)
    x = _lsr(draw64(seed, 400, u), 11)
    deg = torch.clamp(torch.searchsorted(thr, x, right=True), min=1)
    total = int(deg.sum().item())
    left = torch.repeat_interleave(u, deg)
    right = draw_int(seed, 401, torch.arange(total, device=dev, dtype=torch.int64), 0, nr - 1)
    key = torch.unique(left * nr + right)
    left, right = key // nr, key % nr
    s, t = nl + nr, nl + nr + 1
    src = torch.cat([left, torch.full((nl,), s, device=dev, dtype=torch.int64),
                     torch.arange(nl, nl + nr, device=dev, dtype=torch.int64)])
    dst = torch.cat([nl + right, torch.arange(nl, device=dev, dtype=torch.int64),
                     torch.full((nr,), t, device=dev, dtype=torch.int64)])
    cap = torch.ones(src.numel(), device=dev, dtype=torch.int32)
    return FlowInstance(f"bip{nl}x{nr}d{mean_degree}", nl + nr + 2, src.int(), dst.int(), cap,
                        s, t, {"nl": nl, "nr": nr, "mean_degree": mean_degree, "seed": seed})


# --------------------------------------------------------------------------
# Batch mix: instance i uses seed base_seed + i.  With probability 1/2 a
# grid whose side is a log-uniform integer in [grid_lo, grid_hi] (caps
# U[1,255], terminal arcs 2550), else a Poisson bipartite graph whose side is
# a log-uniform integer in [bip_lo, bip_hi] with mean degree U{4..16}.
# --------------------------------------------------------------------------
def batch_spec(count: int, base_seed: int = 1000, grid_lo=32, grid_hi=512,
               bip_lo=1 << 10, bip_hi=1 << 18):
    specs = []
    for i in range(count):
        sd = base_seed + i
        ctr = torch.arange(4, dtype=torch.int64)
        r = draw64(sd, 500, ctr)
        u = [(int(x) & ((1 << 53) - 1)) / float(1 << 53) for x in _lsr(r, 11).tolist()]
        if u[0] < 0.5:
            side = int(math.floor(math.exp(math.log(grid_lo) + u[1] * (math.log(grid_hi + 1) - math.log(grid_lo)))))
            side = min(max(side, grid_lo), grid_hi)
            specs.append(("grid", side, sd))
        else:
            side = int(math.floor(math.exp(math.log(bip_lo) + u[1] * (math.log(bip_hi + 1) - math.log(bip_lo)))))
            side = min(max(side, bip_lo), bip_hi)
            deg = 4 + int(u[2] * 13)
            specs.append(("bip", side, deg, sd))
    return specs


def make_from_spec(spec, device="cpu") -> FlowInstance:
    if spec[0] == "grid":
        _, side, sd = spec
        return grid(side, side, sd, 1, 255, 2550, device=device)
    _, side, deg, sd = spec
    return bipartite_poisson(side, side, deg, sd, device=device)


# --------------------------------------------------------------------------
# Small random graphs for exhaustive tests.
# --------------------------------------------------------------------------
def random_small(n: int, m: int, seed: int, cap_lo: int = 0, cap_hi: int = 10,
                 allow_loops: bool = True) -> FlowInstance:
    ctr = torch.arange(m, dtype=torch.int64)
    src = draw_int(seed, 600, ctr, 0, n - 1)
    dst = draw_int(seed, 601, ctr, 0, n - 1)
    if not allow_loops:
        dst = torch.where(dst == src, (dst + 1) % n, dst)
    cap = draw_int(seed, 602, ctr, cap_lo, cap_hi)
    st = draw_int(seed, 603, torch.arange(2, dtype=torch.int64), 0, n - 1).tolist()
    s, t = st[0], st[1]
    if s == t:
        t = (s + 1) % n
    return FlowInstance(f"rand{n}x{m}", n, src.int(), dst.int(), cap.int(), s, t, {"seed": seed})
