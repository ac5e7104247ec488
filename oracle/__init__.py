"""CPU oracle for maximum flow / minimum cut.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
imports nothing from the CUDA library.

The arithmetic lives in ``maxflow_oracle.c`` (plain C, single-threaded,
exact int64).  This module only compiles it with gcc and marshals numpy
arrays through ctypes.  What each routine follows:

* ``maxflow_pr``   -- FIFO push-relabel with global relabel and gap
  heuristic, paper §2.2 (sequential form of the procedure of Alg. 1), plus a
  second phase that returns stranded excess to s.
* ``maxflow_dinic`` -- Dinic's algorithm (paper §2.1, background).
* ``mincut_brute`` -- the definition of §2.1 by enumerating every s-t cut.
* ``matching_hk``  -- Hopcroft-Karp bipartite matching (§4.1 matching task).
* ``verify_flow``  -- capacity, conservation, value and cut certificate.
* ``residual_dist`` -- global-relabel heights (§2.2) of a residual snapshot.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "maxflow_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

OK, EINVAL, ENOMEM, EINTERNAL = 0, -1, -2, -3


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("arcs_scanned", ctypes.c_int64),
        ("pushes", ctypes.c_int64),
        ("relabels", ctypes.c_int64),
        ("global_relabels", ctypes.c_int64),
        ("gaps", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2)."""
    with _LOCK:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
        return _SO


def _lib():
    global _LIB
    if _LIB is None:
        # ORACLE_SO lets the oracle's own mutation tests load a deliberately
        # broken build of maxflow_oracle.c in a child process.
        lib = ctypes.CDLL(os.environ.get("ORACLE_SO") or build())
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        lib.oracle_maxflow_pr.argtypes = [i64, i64, p, p, p, i32, i32, p, p, p, p]
        lib.oracle_maxflow_dinic.argtypes = [i64, i64, p, p, p, i32, i32, p, p]
        lib.oracle_mincut_brute.argtypes = [i64, i64, p, p, p, i32, i32, p, p]
        lib.oracle_matching_hk.argtypes = [i64, i64, i64, p, p, p]
        lib.oracle_verify_flow.argtypes = [i64, i64, p, p, p, i32, i32, p, i64, p, p]
        lib.oracle_residual_dist.argtypes = [i64, i64, p, p, p, i32, i32, i32, i32, i32, p]
        for f in (lib.oracle_maxflow_pr, lib.oracle_maxflow_dinic, lib.oracle_mincut_brute,
                  lib.oracle_matching_hk, lib.oracle_verify_flow, lib.oracle_residual_dist):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _arr(x, dtype):
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else ctypes.c_void_p(0)


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def maxflow_pr(n, src, dst, cap, s, t, want_flow=True, want_cut=True):
    """FIFO push-relabel.  Returns dict(value, flow, source_side, stats)."""
    src, dst, cap = _arr(src, np.int32), _arr(dst, np.int32), _arr(cap, np.int32)
    m = src.size
    value = ctypes.c_int64(0)
    flow = np.zeros(m, np.int32) if want_flow else None
    side = np.zeros(n, np.uint8) if want_cut else None
    st = OracleStats()
    rc = _lib().oracle_maxflow_pr(
        n, m, _ptr(src), _ptr(dst), _ptr(cap), int(s), int(t), ctypes.byref(value),
        _ptr(flow) if flow is not None else None, _ptr(side) if side is not None else None,
        ctypes.byref(st))
    _check(rc, "maxflow_pr")
    stats = {k: getattr(st, k) for k, _ in OracleStats._fields_}
    return {"value": value.value, "flow": flow, "source_side": side, "stats": stats}


def maxflow_dinic(n, src, dst, cap, s, t, want_flow=False):
    src, dst, cap = _arr(src, np.int32), _arr(dst, np.int32), _arr(cap, np.int32)
    m = src.size
    value = ctypes.c_int64(0)
    flow = np.zeros(m, np.int32) if want_flow else None
    rc = _lib().oracle_maxflow_dinic(
        n, m, _ptr(src), _ptr(dst), _ptr(cap), int(s), int(t), ctypes.byref(value),
        _ptr(flow) if flow is not None else None)
    _check(rc, "maxflow_dinic")
    return {"value": value.value, "flow": flow}


def mincut_brute(n, src, dst, cap, s, t):
    """Minimum cut by enumeration (n <= 22): (value, minimal source side)."""
    src, dst, cap = _arr(src, np.int32), _arr(dst, np.int32), _arr(cap, np.int32)
    value = ctypes.c_int64(0)
    side = np.zeros(n, np.uint8)
    rc = _lib().oracle_mincut_brute(n, src.size, _ptr(src), _ptr(dst), _ptr(cap), int(s),
                                    int(t), ctypes.byref(value), _ptr(side))
    _check(rc, "mincut_brute")
    return value.value, side


def matching_hk(nl, nr, eu, ev):
    eu, ev = _arr(eu, np.int32), _arr(ev, np.int32)
    size = ctypes.c_int64(0)
    rc = _lib().oracle_matching_hk(nl, nr, eu.size, _ptr(eu), _ptr(ev), ctypes.byref(size))
    _check(rc, "matching_hk")
    return size.value


def verify_flow(n, src, dst, cap, s, t, flow, value):
    """Returns (code, cut_capacity, source_side); code 0 = certified maximum flow."""
    src, dst, cap = _arr(src, np.int32), _arr(dst, np.int32), _arr(cap, np.int32)
    flow = _arr(flow, np.int32)
    cut = ctypes.c_int64(-1)
    side = np.zeros(n, np.uint8)
    rc = _lib().oracle_verify_flow(n, src.size, _ptr(src), _ptr(dst), _ptr(cap), int(s),
                                   int(t), _ptr(flow), int(value), ctypes.byref(cut),
                                   _ptr(side))
    if rc < 0:
        _check(rc, "verify_flow")
    return rc, cut.value, side


def residual_dist(n, tail, head, rescap, target, excluded, base, unreach, excluded_h):
    tail, head = _arr(tail, np.int32), _arr(head, np.int32)
    rescap = _arr(rescap, np.int64)
    dist = np.zeros(n, np.int32)
    rc = _lib().oracle_residual_dist(n, tail.size, _ptr(tail), _ptr(head), _ptr(rescap),
                                     int(target), int(excluded), int(base), int(unreach),
                                     int(excluded_h), _ptr(dist))
    _check(rc, "residual_dist")
    return dist
