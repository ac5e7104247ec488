"""The residual layouts of paper §3.2 (Fig. 2) written out by definition.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

bcsr(): for every vertex u, the neighbours v joined to u by an arc in either
direction (self-loops ignored), sorted by id; the slot of (u, v) holds the
initial residual capacity c(u,v) = sum of the capacities of the arcs u -> v,
and rev gives the slot of (v, u).  arc2slot maps every input arc to the slot
of (src, dst), or 2^32 - 1 for a self-loop.

rcsr(): out rows = the non-loop arcs ordered by (src, dst, input position),
holding head and capacity; in rows = the same arcs ordered by (dst, src,
out slot), holding the tail and flow_idx, the out slot of the arc.
"""
import numpy as np

NONE = np.uint32(0xFFFFFFFF)


def _offsets(rows, n):
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, rows + 1, 1)
    return np.cumsum(off)


def bcsr(n, src, dst, cap):
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    cap = np.asarray(cap, np.int64)
    keep = src != dst
    u, v, c = src[keep], dst[keep], cap[keep]
    keys = np.concatenate([u * n + v, v * n + u])
    vals = np.concatenate([c, np.zeros_like(c)])
    ukeys, inv = np.unique(keys, return_inverse=True)
    cf0 = np.zeros(ukeys.size, np.int64)
    np.add.at(cf0, inv, vals)
    rows = ukeys // n
    col = (ukeys % n).astype(np.int32)
    off = _offsets(rows, n)
    rev = np.searchsorted(ukeys, col.astype(np.int64) * n + rows).astype(np.uint32)
    arc2slot = np.full(src.size, NONE, np.uint32)
    arc2slot[keep] = np.searchsorted(ukeys, u * n + v).astype(np.uint32)
    return {"offsets": off, "col": col, "cap": cf0.astype(np.int32), "rev": rev,
            "arc2slot": arc2slot}


def rcsr(n, src, dst, cap):
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    cap = np.asarray(cap, np.int64)
    idx = np.nonzero(src != dst)[0]
    order = idx[np.lexsort((idx, dst[idx], src[idx]))]
    col = dst[order].astype(np.int32)
    capo = cap[order].astype(np.int32)
    off = _offsets(src[order], n)
    arc2slot = np.full(src.size, NONE, np.uint32)
    arc2slot[order] = np.arange(order.size, dtype=np.uint32)
    j = np.arange(order.size)
    tails = src[order]
    inorder = np.lexsort((j, tails, dst[order]))
    in_col = tails[inorder].astype(np.int32)
    flow_idx = inorder.astype(np.uint32)
    in_off = _offsets(dst[order][inorder], n)
    return {"offsets": off, "col": col, "cap": capo, "arc2slot": arc2slot,
            "in_offsets": in_off, "in_col": in_col, "flow_idx": flow_idx}
