"""Python binding of the WBPR C ABI (``include/wbpr.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libwbpr.so``.  Functions keep the C names.  Arrays may be
torch tensors (host or CUDA) or numpy arrays; streams are torch streams,
raw ``cudaStream_t`` integers, or None (legacy default stream).

If the library is missing or cannot be loaded, every call raises
``RuntimeError``: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "WBPR_RCSR", "WBPR_BCSR", "WbprError", "Options", "Stats", "Info", "Graph", "load",
    "wbpr_build", "wbpr_maxflow", "wbpr_maxflow_async", "wbpr_solve_status", "wbpr_mincut",
    "wbpr_maxflow_batch", "wbpr_destroy", "wbpr_default_options", "wbpr_get_options",
    "wbpr_set_options", "wbpr_get_stats", "wbpr_get_info", "wbpr_last_error",
    "wbpr_last_error_message", "wbpr_error_string", "wbpr_run_stage", "wbpr_export",
    "use_torch_allocator", "EXPORTED_SYMBOLS",
]

WBPR_RCSR, WBPR_BCSR = 0, 1
STATUS = {0: "WBPR_OK", -1: "WBPR_EINVAL", -2: "WBPR_ENOMEM", -3: "WBPR_ECUDA",
          -4: "WBPR_ETIMEOUT", -5: "WBPR_EOVERFLOW", -6: "WBPR_ESTATE"}
STAGE_PREFLOW, STAGE_GLOBAL_RELABEL, STAGE_ITERATIONS = 1, 2, 3
ARRAY = {"height": (1, np.int32), "excess": (2, np.int64), "offsets": (3, np.int64),
         "col": (4, np.int32), "cf": (5, np.int32), "cap": (6, np.int32), "rev": (7, np.uint32),
         "bf": (8, np.int32), "in_offsets": (9, np.int64), "in_col": (10, np.int32),
         "flow_idx": (11, np.uint32), "arc2slot": (12, np.uint32), "excess_total": (13, np.int64),
         "trace": (14, np.uint64), "trace_len": (15, np.uint32), "order": (16, np.int32),
         "st": (17, np.int32), "warp_time": (18, np.uint64)}

# Every function declared in include/wbpr.h.
EXPORTED_SYMBOLS = [
    "wbpr_build", "wbpr_build_ex", "wbpr_maxflow", "wbpr_maxflow_async", "wbpr_solve_status",
    "wbpr_mincut", "wbpr_maxflow_batch", "wbpr_destroy", "wbpr_default_options",
    "wbpr_get_options", "wbpr_set_options", "wbpr_get_stats", "wbpr_get_info",
    "wbpr_last_error", "wbpr_last_error_message", "wbpr_error_string", "wbpr_set_allocator",
    "wbpr_run_stage", "wbpr_export", "wbpr_maxflow_bcsr_noalloc",
    "wbpr_server_default_options", "wbpr_server_start", "wbpr_server_submit", "wbpr_server_poll",
    "wbpr_server_stop", "wbpr_server_team_exits", "wbpr_server_times",
]


class WbprError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("use_rev", ctypes.c_int32), ("gap", ctypes.c_int32),
                ("multi_push", ctypes.c_int32), ("cycle", ctypes.c_int32),
                ("small_max_degree", ctypes.c_int32), ("small_tile", ctypes.c_int32),
                ("warp_max_degree", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("barrier_timeout_ms", ctypes.c_int32), ("max_iterations", ctypes.c_int64),
                ("trace", ctypes.c_int32), ("gr_ratio", ctypes.c_float),
                ("batch_team", ctypes.c_int32), ("batch_big_slots", ctypes.c_int64),
                ("bottom_up", ctypes.c_int32), ("bottom_up_min", ctypes.c_int32),
                ("renumber", ctypes.c_int32), ("thread_centric", ctypes.c_int32),
                ("warp_time", ctypes.c_int32), ("stage_hubs", ctypes.c_int32),
                ("barrier_extra", ctypes.c_int32), ("bottom_up_edges", ctypes.c_int32),
                ("avq_incremental", ctypes.c_int32), ("lean_build", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("phase1_iterations", ctypes.c_int64),
                ("global_relabels", ctypes.c_int64), ("active_total", ctypes.c_int64),
                ("arcs_scanned", ctypes.c_int64), ("gr_arcs_scanned", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("relabels", ctypes.c_int64), ("gaps", ctypes.c_int64),
                ("written_off", ctypes.c_int64), ("solve_ms", ctypes.c_double),
                ("avq_full_scans", ctypes.c_int64), ("avq_bitmap_scans", ctypes.c_int64),
                ("avq_candidates", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("s", ctypes.c_int32),
                ("t", ctypes.c_int32), ("layout", ctypes.c_int32), ("slots", ctypes.c_int64),
                ("max_degree", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("grid_blocks", ctypes.c_int32), ("num_sms", ctypes.c_int32),
                ("renumbered", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_LOCK = threading.Lock()
_ALLOC_CBS = None
_P = ctypes.c_void_p
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libwbpr.so (optionally compiling it first)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"WBPR CUDA library not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.wbpr_build.argtypes = [i64, i64, _P, _P, _P, i32, i32, i32]
        lib.wbpr_build.restype = _P
        lib.wbpr_build_ex.argtypes = [i64, i64, _P, _P, _P, i32, i32, i32, _P, _P]
        lib.wbpr_build_ex.restype = _P
        lib.wbpr_maxflow.argtypes = [_P, _P, _P, _P]
        lib.wbpr_maxflow_async.argtypes = [_P, _P, _P, _P]
        lib.wbpr_solve_status.argtypes = [_P, _P]
        lib.wbpr_mincut.argtypes = [_P, _P, _P, _P]
        lib.wbpr_maxflow_batch.argtypes = [_P, i32, _P, _P, _P]
        lib.wbpr_destroy.argtypes = [_P]
        lib.wbpr_destroy.restype = None
        lib.wbpr_default_options.argtypes = [_P]
        lib.wbpr_default_options.restype = None
        lib.wbpr_get_options.argtypes = [_P, _P]
        lib.wbpr_set_options.argtypes = [_P, _P]
        lib.wbpr_get_stats.argtypes = [_P, _P]
        lib.wbpr_get_info.argtypes = [_P, _P]
        lib.wbpr_last_error.argtypes = []
        lib.wbpr_last_error_message.argtypes = []
        lib.wbpr_last_error_message.restype = ctypes.c_char_p
        lib.wbpr_error_string.argtypes = [i32]
        lib.wbpr_error_string.restype = ctypes.c_char_p
        lib.wbpr_set_allocator.argtypes = [_P, _P, _P]
        lib.wbpr_run_stage.argtypes = [_P, _P, i32, i64]
        lib.wbpr_export.argtypes = [_P, i32, _P, i64]
        lib.wbpr_maxflow_bcsr_noalloc.argtypes = [i32, i64, i32, i32, _P, _P, _P, _P, _P, _P, _P]
        lib.wbpr_server_default_options.argtypes = [_P]
        lib.wbpr_server_default_options.restype = None
        lib.wbpr_server_start.argtypes = [_P]
        lib.wbpr_server_start.restype = _P
        lib.wbpr_server_submit.argtypes = [_P, _P]
        lib.wbpr_server_submit.restype = i64
        lib.wbpr_server_poll.argtypes = [_P, i64, _P]
        lib.wbpr_server_stop.argtypes = [_P]
        lib.wbpr_server_team_exits.argtypes = [_P, _P, i32]
        lib.wbpr_server_times.argtypes = [_P, i64, _P, _P]
        for name in ("wbpr_maxflow", "wbpr_maxflow_async", "wbpr_solve_status", "wbpr_mincut",
                     "wbpr_maxflow_batch", "wbpr_get_options", "wbpr_set_options",
                     "wbpr_get_stats", "wbpr_get_info", "wbpr_last_error", "wbpr_set_allocator",
                     "wbpr_run_stage", "wbpr_export", "wbpr_maxflow_bcsr_noalloc", "wbpr_server_poll",
                     "wbpr_server_stop", "wbpr_server_team_exits", "wbpr_server_times"):
            getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
        return lib


def _check(rc: int):
    if rc != 0:
        lib = load()
        raise WbprError(rc, (lib.wbpr_last_error_message() or b"").decode())


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class _Buf:
    """Pointer to a torch tensor or numpy array (kept alive by this object)."""

    def __init__(self, x, dtype):
        self.keep = None
        if x is None:
            self.ptr = None
            return
        try:
            import torch
            if isinstance(x, torch.Tensor):
                tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
                if x.dtype != tdt:
                    raise TypeError(f"expected {tdt}, got {x.dtype}")
                if not x.is_contiguous():
                    raise ValueError("tensor must be contiguous")
                self.keep = x
                self.ptr = x.data_ptr() if x.numel() else None
                return
        except ImportError:
            pass
        a = np.ascontiguousarray(x, dtype=dtype)
        self.keep = a
        self.ptr = a.ctypes.data if a.size else None


class Graph:
    """Owns one wbpr_graph handle."""

    def __init__(self, handle: int, n: int, m: int, s: int, t: int, layout: int):
        self.handle = handle
        self.n, self.m, self.s, self.t, self.layout = n, m, s, t, layout

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            load().wbpr_destroy(self.handle)
            self.handle = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _ALLOC_CBS
    lib = load()
    if not enable:
        _check(lib.wbpr_set_allocator(None, None, None))
        _ALLOC_CBS = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(lib.wbpr_set_allocator(ctypes.cast(cbs[0], _P), ctypes.cast(cbs[1], _P), None))
    _ALLOC_CBS = cbs


def torch_allocator_enabled() -> bool:
    return _ALLOC_CBS is not None


def wbpr_default_options() -> Options:
    o = Options()
    load().wbpr_default_options(ctypes.byref(o))
    return o


def wbpr_build(n, m, src, dst, cap, s, t, layout=WBPR_BCSR, opts: Options | None = None,
               stream=None) -> Graph:
    lib = load()
    bs, bd, bc = _Buf(src, np.int32), _Buf(dst, np.int32), _Buf(cap, np.int32)
    h = lib.wbpr_build_ex(int(n), int(m), bs.ptr, bd.ptr, bc.ptr, int(s), int(t), int(layout),
                          ctypes.byref(opts) if opts is not None else None, _stream(stream))
    if not h:
        raise WbprError(lib.wbpr_last_error(), (lib.wbpr_last_error_message() or b"").decode())
    return Graph(h, int(n), int(m), int(s), int(t), int(layout))


def wbpr_maxflow(g: Graph, stream=None, edge_flow=None) -> int:
    v = ctypes.c_int64(0)
    b = _Buf(edge_flow, np.int32)
    _check(load().wbpr_maxflow(g.handle, _stream(stream), ctypes.byref(v), b.ptr))
    return v.value


def wbpr_maxflow_async(g: Graph, stream, d_value, d_edge_flow=None) -> None:
    bv, be = _Buf(d_value, np.int64), _Buf(d_edge_flow, np.int32)
    _check(load().wbpr_maxflow_async(g.handle, _stream(stream), bv.ptr, be.ptr))


def wbpr_solve_status(g: Graph, stream=None) -> None:
    _check(load().wbpr_solve_status(g.handle, _stream(stream)))


def wbpr_mincut(g: Graph, stream=None, source_side=None) -> int:
    v = ctypes.c_int64(0)
    b = _Buf(source_side, np.uint8)
    _check(load().wbpr_mincut(g.handle, _stream(stream), ctypes.byref(v), b.ptr))
    return v.value


def wbpr_maxflow_batch(gs, stream=None, edge_flows=None):
    count = len(gs)
    handles = (ctypes.c_void_p * max(1, count))(*[x.handle for x in gs])
    values = (ctypes.c_int64 * max(1, count))()
    keep = []
    flows = None
    if edge_flows is not None:
        bufs = [_Buf(f, np.int32) for f in edge_flows]
        keep.extend(bufs)
        flows = (ctypes.c_void_p * max(1, count))(*[b.ptr for b in bufs])
    _check(load().wbpr_maxflow_batch(handles, count, _stream(stream), values, flows))
    return [values[i] for i in range(count)]


def wbpr_destroy(g: Graph) -> None:
    g.close()


def wbpr_get_options(g: Graph) -> Options:
    o = Options()
    _check(load().wbpr_get_options(g.handle, ctypes.byref(o)))
    return o


def wbpr_set_options(g: Graph, opts: Options) -> None:
    _check(load().wbpr_set_options(g.handle, ctypes.byref(opts)))


def wbpr_get_stats(g: Graph) -> dict:
    s = Stats()
    _check(load().wbpr_get_stats(g.handle, ctypes.byref(s)))
    return s.as_dict()


def wbpr_get_info(g: Graph) -> dict:
    i = Info()
    _check(load().wbpr_get_info(g.handle, ctypes.byref(i)))
    return i.as_dict()


def wbpr_last_error() -> int:
    return load().wbpr_last_error()


def wbpr_last_error_message() -> str:
    return (load().wbpr_last_error_message() or b"").decode()


def wbpr_error_string(status: int) -> str:
    return (load().wbpr_error_string(int(status)) or b"").decode()


def wbpr_run_stage(g: Graph, stage: int, arg: int = 0, stream=None) -> None:
    _check(load().wbpr_run_stage(g.handle, _stream(stream), int(stage), int(arg)))


def wbpr_export(g: Graph, what: str, count: int | None = None) -> np.ndarray:
    code, dt = ARRAY[what]
    if count is None:
        info = wbpr_get_info(g)
        count = {"height": info["n"], "excess": info["n"], "offsets": info["n"] + 1,
                 "in_offsets": info["n"] + 1, "arc2slot": info["m"], "excess_total": 1,
                 "order": info["n"] if info["renumbered"] else 0, "st": 2,
                 "warp_time": 8 * info["grid_blocks"] if wbpr_get_options(g).warp_time else 0}.get(
                     what, info["slots"])
    if what == "trace":
        length = wbpr_export(g, "trace_len", 1)[0] if wbpr_get_options(g).trace > 0 else 0
        out = np.zeros(4 * int(length), dtype=dt)
        _check(load().wbpr_export(g.handle, code, out.ctypes.data if length else None, out.size))
        return out.reshape(-1, 4)
    out = np.zeros(count, dtype=dt)
    _check(load().wbpr_export(g.handle, code, out.ctypes.data if count else None, int(count)))
    return out


NOALLOC_MAX_VERTICES = 65536
NOALLOC_MAX_SLOTS = 1048576


def wbpr_maxflow_bcsr_noalloc(n, slots, s, t, off, col, cap, rev, stream=None, d_value=None,
                              d_residual=None) -> None:
    """Allocation-free solve of a BCSR graph held in device tensors (see wbpr.h).

    off int64[n+1], col int32[slots], cap int32[slots], rev int32[slots] (the
    uint32 reverse slots viewed as int32), d_value int64[1] and optional
    d_residual int32[slots], all on the current CUDA device."""
    bo, bc, bk = _Buf(off, np.int64), _Buf(col, np.int32), _Buf(cap, np.int32)
    br, bv, bres = _Buf(rev, np.int32), _Buf(d_value, np.int64), _Buf(d_residual, np.int32)
    _check(load().wbpr_maxflow_bcsr_noalloc(int(n), int(slots), int(s), int(t), bo.ptr, bc.ptr, bk.ptr,
                                            br.ptr, _stream(stream), bv.ptr, bres.ptr))


class ServerOptions(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("capacity", ctypes.c_int32), ("team_blocks", ctypes.c_int32),
                ("big_teams", ctypes.c_int32), ("small_blocks", ctypes.c_int32), ("idle_ms", ctypes.c_int32),
                ("big_slots", ctypes.c_int64), ("build_room", ctypes.c_int32)]


def wbpr_server_default_options() -> ServerOptions:
    o = ServerOptions()
    load().wbpr_server_default_options(ctypes.byref(o))
    return o


def wbpr_server_start(opts: ServerOptions | None = None) -> int:
    lib = load()
    h = lib.wbpr_server_start(ctypes.byref(opts) if opts is not None else None)
    if not h:
        raise WbprError(lib.wbpr_last_error(), (lib.wbpr_last_error_message() or b"").decode())
    return h


def wbpr_server_submit(server: int, g: Graph) -> int:
    t = load().wbpr_server_submit(server, g.handle)
    if t < 0:
        _check(int(t))
    return int(t)


def wbpr_server_poll(server: int, ticket: int):
    """The flow value once the request is done, else None."""
    v = ctypes.c_int64(0)
    rc = load().wbpr_server_poll(server, int(ticket), ctypes.byref(v))
    if rc == 1:
        return None
    _check(rc)
    return v.value


def wbpr_server_times(server: int, ticket: int):
    """(start, end) of a finished request on the device's globaltimer in ns,
    else None while it is pending."""
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = load().wbpr_server_times(server, int(ticket), ctypes.byref(a), ctypes.byref(b))
    if rc == 1:
        return None
    _check(rc)
    return a.value, b.value


def wbpr_server_stop(server: int) -> None:
    _check(load().wbpr_server_stop(server))


def wbpr_server_team_exits(server: int, count: int):
    """Exit reason per team once the server kernel has ended, else None."""
    out = (ctypes.c_int32 * max(1, count))()
    rc = load().wbpr_server_team_exits(server, out, int(count))
    if rc == 1:
        return None
    _check(rc)
    return list(out)[:count]
