"""s-line graphs of non-uniform hypergraphs on GB300: Python binding of libslg.

Argument marshalling only: each function below calls the C entry point of the
same name in ``libslg.so`` (declared in ``include/slg.h``), and every step of
the computation runs in that library's CUDA kernels. Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); torch is used for device memory
and streams only. There is no CPU fallback: if the library is missing, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "SlgError", "Graph", "slg_load", "slg_free", "slg_count", "slg_bound", "slg_build",
    "slg_build_window", "slg_plan_windows", "slg_row_offsets", "slg_transpose_copy",
    "slg_graph_info", "slg_set_timing", "slg_last_timing", "slg_set_bins", "slg_kernel_stats",
    "slg_mode_stats", "slg_ensemble_mode_stats", "slg_kernel_launches", "slg_scan_counts_noalloc", "slg_batch_load",
    "slg_batch_info", "slg_batch_pair_offsets", "slg_batch", "slg_result_free", "slg_dual", "slg_ensemble_count",
    "slg_ensemble_row_offsets", "slg_ensemble_plan_windows", "slg_ensemble_build_window",
    "slg_ensemble_build", "ENSEMBLE_MAX", "ENSEMBLE_ALL", "slg_autotune", "slg_set_hub_pairs", "slg_set_staging", "slg_staging_stats", "slg_set_ensemble_filter", "slg_ensemble_fill_stats",
    "slg_stream_window", "slg_ensemble_stream_window",
    "Server", "slg_serve_create", "slg_serve_destroy",
    "slg_serve_register", "slg_serve_submit", "slg_serve_poll", "slg_serve_fetch",
    "slg_serve_release", "slg_serve_stats", "library_path",
    "lib",
]

SLG_OK = 0
SLG_EINVAL = 1
SLG_ENOMEM = 2
SLG_ECUDA = 3
SLG_ETIMEOUT = 4
SLG_ECAPACITY = 5
SLG_EBUSY = 6
SLG_EINTERNAL = 7
_NAMES = {0: "SLG_OK", 1: "SLG_EINVAL", 2: "SLG_ENOMEM", 3: "SLG_ECUDA", 4: "SLG_ETIMEOUT",
          5: "SLG_ECAPACITY", 6: "SLG_EBUSY", 7: "SLG_EINTERNAL"}


class SlgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)

class BatchResult(ctypes.Structure):
    _fields_ = [("want_list", ctypes.c_int32), ("status", ctypes.c_int32),
                ("pairs", ctypes.c_int64), ("wedges", ctypes.c_int64),
                ("digest", ctypes.c_uint64), ("I", _i32p), ("J", _i32p), ("O", _i32p)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("window_pairs", ctypes.c_int64),
                ("max_result_pairs", ctypes.c_int64), ("workers", ctypes.c_int32),
                ("max_s", ctypes.c_int32), ("digest", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("small_workers", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("small_wedges", ctypes.c_int64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("materialized", ctypes.c_int32),
                ("pairs", ctypes.c_int64), ("wedges", ctypes.c_int64),
                ("digest", ctypes.c_uint64), ("latency_us", ctypes.c_double),
                ("queue_us", ctypes.c_double), ("batch_size", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("span_s", ctypes.c_double),
                ("queries_per_s", ctypes.c_double), ("pairs_per_s", ctypes.c_double),
                ("wedges_per_s", ctypes.c_double), ("peak_memory", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("running", ctypes.c_int64),
                ("batched", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batch_overflows", ctypes.c_int64), ("batch_failures", ctypes.c_int64)]


_SIGS = {
    "slg_last_error": (ctypes.c_char_p, []),
    "slg_version": (_i32, []),
    "slg_load": (_i32, [_vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "slg_free": (None, [_vp]),
    "slg_graph_info": (_i32, [_vp, _i32p, _i32p, _i64p]),
    "slg_transpose_copy": (_i32, [_vp, _vp, _vp]),
    "slg_count": (_i32, [_vp, _i32, _i64p, _i64p]),
    "slg_bound": (_i32, [_vp, _i32, _i64p]),
    "slg_row_offsets": (_i32, [_vp, _i32, _vp]),
    "slg_build": (_i32, [_vp, _i32, _vp, _vp, _vp, _i64, _i64p]),
    "slg_build_window": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _i64, _i64p, _u64p, _vp]),
    "slg_plan_windows": (_i32, [_vp, _i32, _i64, _i32p, _i32, _i32p]),
    "slg_ensemble_count": (_i32, [_vp, _i32p, _i32, _i64p, _i64p]),
    "slg_ensemble_row_offsets": (_i32, [_vp, _i32p, _i32, _vp]),
    "slg_ensemble_plan_windows": (_i32, [_vp, _i32p, _i32, _i32, _i64, _i32p, _i32, _i32p]),
    "slg_ensemble_build_window": (_i32, [_vp, _i32p, _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                         _i64, _i64p, _u64p, _vp]),
    "slg_ensemble_stream_window": (_i32, [_vp, _i32p, _i32, _i32, _vp, _vp, _vp, _i64, _i32p,
                                          _i64p]),
    "slg_stream_window": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, _i64, _i32p, _i64p]),
    "slg_set_timing": (_i32, [_vp, _i32]),
    "slg_last_timing": (_i32, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "slg_set_bins": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _i32]),
    "slg_set_hub_pairs": (_i32, [_vp, _i32, _i64]),
    "slg_set_staging": (_i32, [_vp, _i64]),
    "slg_set_ensemble_filter": (_i32, [_vp, _i32]),
    "slg_staging_stats": (_i32, [_vp, _i64p]),
    "slg_ensemble_fill_stats": (_i32, [_vp, _i32, _i64p]),
    "slg_autotune": (_i32, [_vp, _i32, _i32, _i32p, ctypes.POINTER(ctypes.c_float)]),
    "slg_kernel_stats": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_float), _i64p]),
    "slg_mode_stats": (_i32, [_vp, _i32, _i64p]),
    "slg_ensemble_mode_stats": (_i32, [_vp, _i32p, _i32, _i32, _i64p]),
    "slg_kernel_launches": (_i64, []),
    "slg_scan_counts_noalloc": (_i32, [_vp, _vp, _i64, _vp]),
    "slg_batch_load": (_i32, [ctypes.POINTER(_vp), _i32p, _i32, _vp, ctypes.POINTER(_vp)]),
    "slg_dual": (_i32, [_vp, _vp, ctypes.POINTER(_vp)]),
    "slg_batch_info": (_i32, [_vp, _i32p, _i32p]),
    "slg_batch_pair_offsets": (_i32, [_vp, _i64p]),
    "slg_batch": (_i32, [ctypes.POINTER(_vp), _i32p, _i32, ctypes.POINTER(BatchResult)]),
    "slg_result_free": (None, [ctypes.POINTER(BatchResult)]),
    "slg_serve_create": (_i32, [ctypes.POINTER(ServeCfg), ctypes.POINTER(_vp)]),
    "slg_serve_destroy": (None, [_vp]),
    "slg_serve_register": (_i32, [_vp, _vp, _i32p]),
    "slg_serve_submit": (_i32, [_vp, _i32, _i32, ctypes.POINTER(ctypes.c_uint64)]),
    "slg_serve_poll": (_i32, [_vp, ctypes.c_uint64, _i32, ctypes.POINTER(ServeResult)]),
    "slg_serve_fetch": (_i32, [_vp, ctypes.c_uint64, _vp, _vp, _vp, _i64]),
    "slg_serve_release": (_i32, [_vp, ctypes.c_uint64]),
    "slg_serve_stats": (_i32, [_vp, _i32, ctypes.POINTER(ServeStats)]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libslg (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libslg is not built ({path} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(code: int):
    if code != SLG_OK:
        raise SlgError(code, (lib().slg_last_error() or b"").decode())


def _ptr(a) -> int:
    """Data pointer of a contiguous int array (numpy or torch) or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_handle(stream) -> int:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Graph:
    """A hypergraph resident on the GPU (handle of libslg)."""

    def __init__(self, handle: int, m: int, n: int, nnz: int, keep=None):
        self._h = handle
        self.m, self.n, self.nnz = m, n, nnz
        self._keep = keep

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("graph was freed")
        return self._h

    def free(self):
        if self._h:
            lib().slg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _as_i32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.int32)
    import torch
    if a.dtype != torch.int32:
        raise TypeError("CSR arrays must be int32")
    return a.contiguous()


def slg_load(off, idx, m: int, n: int, stream=None) -> Graph:
    off = _as_i32(off)
    idx = _as_i32(idx)
    h = _vp()
    _check(lib().slg_load(_ptr(off), _ptr(idx) if len(idx) else None, m, n,
                          _stream_handle(stream), ctypes.byref(h)))
    mm, nn, nz = _i32(), _i32(), _i64()
    _check(lib().slg_graph_info(h, ctypes.byref(mm), ctypes.byref(nn), ctypes.byref(nz)))
    return Graph(h.value, mm.value, nn.value, nz.value)


def slg_free(g: Graph):
    g.free()


def slg_graph_info(g: Graph):
    mm, nn, nz = _i32(), _i32(), _i64()
    _check(lib().slg_graph_info(g.handle, ctypes.byref(mm), ctypes.byref(nn), ctypes.byref(nz)))
    return mm.value, nn.value, nz.value


def slg_transpose_copy(g: Graph, offT=None, idxT=None):
    if offT is None:
        offT = np.zeros(g.n + 1, np.int32)
    if idxT is None:
        idxT = np.zeros(max(g.nnz, 1), np.int32)
    _check(lib().slg_transpose_copy(g.handle, _ptr(offT), _ptr(idxT)))
    return offT, idxT[:g.nnz]


def slg_count(g: Graph, s: int):
    """(|L_s|, W_s)."""
    p, w = _i64(), _i64()
    _check(lib().slg_count(g.handle, s, ctypes.byref(p), ctypes.byref(w)))
    return p.value, w.value


def slg_bound(g: Graph, s: int) -> int:
    b = _i64()
    _check(lib().slg_bound(g.handle, s, ctypes.byref(b)))
    return b.value


def slg_row_offsets(g: Graph, s: int, out=None):
    if out is None:
        out = np.zeros(g.m + 1, np.int64)
    _check(lib().slg_row_offsets(g.handle, s, _ptr(out)))
    return out


def slg_build(g: Graph, s: int, I=None, J=None, O=None, cap: int | None = None):
    """The whole edge list of L_s(H). Returns (I, J, O) trimmed to |L_s|.

    Without output arrays, host numpy arrays of the exact size are allocated
    (one counting pass first).
    """
    if I is None:
        pairs, _ = slg_count(g, s)
        I = np.zeros(max(pairs, 1), np.int32)
        J = np.zeros(max(pairs, 1), np.int32)
        O = np.zeros(max(pairs, 1), np.int32)
        cap = pairs
    if cap is None:
        cap = len(I)
    p = _i64()
    _check(lib().slg_build(g.handle, s, _ptr(I), _ptr(J), _ptr(O), cap, ctypes.byref(p)))
    return I[:p.value], J[:p.value], O[:p.value]


def slg_build_window(g: Graph, s: int, row_begin: int, row_end: int, I, J, O,
                     cap: int | None = None, digest: bool = False, row_digests=None):
    """Rows [row_begin, row_end) into I/J/O. Returns (pairs, digest or None)."""
    if cap is None:
        cap = len(I)
    p = _i64()
    d = ctypes.c_uint64()
    _check(lib().slg_build_window(g.handle, s, row_begin, row_end, _ptr(I), _ptr(J), _ptr(O),
                                  cap, ctypes.byref(p), ctypes.byref(d) if digest else None,
                                  _ptr(row_digests)))
    return p.value, (d.value if digest else None)


def slg_plan_windows(g: Graph, s: int, cap: int, max_windows: int = 1 << 20) -> np.ndarray:
    splits = np.zeros(max_windows + 1, np.int32)
    nw = _i32()
    _check(lib().slg_plan_windows(g.handle, s, cap, splits.ctypes.data_as(_i32p), max_windows,
                                  ctypes.byref(nw)))
    return splits[:nw.value + 1].copy()


ENSEMBLE_MAX = 16


def _s_list(s_list):
    a = np.ascontiguousarray(np.asarray(s_list, dtype=np.int32).reshape(-1))
    return a, a.ctypes.data_as(_i32p), int(a.size)


def slg_ensemble_count(g: Graph, s_list):
    """([|L_s| for s in s_list], W_{s_list[0]}); s_list strictly ascending."""
    a, ap, k = _s_list(s_list)
    pairs = np.zeros(max(k, 1), np.int64)
    w = _i64()
    _check(lib().slg_ensemble_count(g.handle, ap, k, pairs.ctypes.data_as(_i64p),
                                    ctypes.byref(w)))
    return [int(x) for x in pairs[:k]], w.value


def slg_ensemble_row_offsets(g: Graph, s_list, out=None):
    """[k, m+1] row offsets, one row per list."""
    a, ap, k = _s_list(s_list)
    if out is None:
        out = np.zeros((k, g.m + 1), np.int64)
    _check(lib().slg_ensemble_row_offsets(g.handle, ap, k, _ptr(out)))
    return out


ENSEMBLE_ALL = -1


def slg_ensemble_plan_windows(g: Graph, s_list, cap: int, which: int = ENSEMBLE_ALL,
                              max_windows: int = 1 << 20) -> np.ndarray:
    """Row splits for windows of at most cap pairs: all lists together (which = -1)
    or list `which` alone."""
    a, ap, k = _s_list(s_list)
    splits = np.zeros(max_windows + 1, np.int32)
    nw = _i32()
    _check(lib().slg_ensemble_plan_windows(g.handle, ap, k, which, cap,
                                           splits.ctypes.data_as(_i32p), max_windows,
                                           ctypes.byref(nw)))
    return splits[:nw.value + 1].copy()


def slg_ensemble_build_window(g: Graph, s_list, row_begin: int, row_end: int, I, J, O,
                              cap: int | None = None, digest: bool = False, row_digests=None,
                              which: int = ENSEMBLE_ALL):
    """Rows [row_begin, row_end) of every list back to back (which = -1) or of list
    `which` alone. Returns (pairs per selected list, digests or None)."""
    a, ap, k = _s_list(s_list)
    if cap is None:
        cap = len(I)
    nl = k if which < 0 else 1
    pairs = np.zeros(max(nl, 1), np.int64)
    dig = np.zeros(max(nl, 1), np.uint64)
    _check(lib().slg_ensemble_build_window(
        g.handle, ap, k, which, row_begin, row_end, _ptr(I), _ptr(J), _ptr(O), cap,
        pairs.ctypes.data_as(_i64p), dig.ctypes.data_as(_u64p) if digest else None,
        _ptr(row_digests)))
    return [int(x) for x in pairs[:nl]], ([int(x) for x in dig[:nl]] if digest else None)


def slg_ensemble_build(g: Graph, s_list):
    """Every list of the ensemble as host arrays: [(I, J, O) per s]."""
    pairs, _ = slg_ensemble_count(g, s_list)
    tot = sum(pairs)
    I = np.zeros(max(tot, 1), np.int32)
    J = np.zeros(max(tot, 1), np.int32)
    O = np.zeros(max(tot, 1), np.int32)
    got, _ = slg_ensemble_build_window(g, s_list, 0, g.m, I, J, O, cap=tot)
    out, b = [], 0
    for p in got:
        out.append((I[b:b + p], J[b:b + p], O[b:b + p]))
        b += p
    return out


def slg_ensemble_stream_window(g: Graph, s_list, row_begin: int, I, J, O,
                               cap: int | None = None):
    """The next one-walk window from row_begin: every list of rows
    [row_begin, row_end) back to back in the device arrays I, J, O.
    Returns (row_end, pairs per list)."""
    a, ap, k = _s_list(s_list)
    if cap is None:
        cap = len(I)
    r1 = _i32()
    pairs = np.zeros(k, np.int64)
    _check(lib().slg_ensemble_stream_window(g.handle, ap, k, row_begin, _ptr(I), _ptr(J), _ptr(O),
                                            cap, ctypes.byref(r1), pairs.ctypes.data_as(_i64p)))
    return int(r1.value), [int(x) for x in pairs]


def slg_stream_window(g: Graph, s: int, row_begin: int, I, J, O, cap: int | None = None):
    """The next one-walk window of L_s from row_begin. Returns (row_end, pairs)."""
    if cap is None:
        cap = len(I)
    r1 = _i32()
    pairs = _i64()
    _check(lib().slg_stream_window(g.handle, s, row_begin, _ptr(I), _ptr(J), _ptr(O), cap,
                                   ctypes.byref(r1), ctypes.byref(pairs)))
    return int(r1.value), int(pairs.value)


def slg_set_timing(g: Graph, enable: bool = True):
    _check(lib().slg_set_timing(g.handle, 1 if enable else 0))


def slg_last_timing(g: Graph):
    ms = (ctypes.c_float * 5)()
    _check(lib().slg_last_timing(g.handle, ms))
    return list(ms)


NMODES = 7
MODE_NAMES = ("warp", "block", "dense", "wdense", "sparse", "wsparse", "hubpair")


def slg_kernel_stats(g: Graph, reset: bool = False):
    """(ms[2][NMODES], launches[2][NMODES]) per pass (count, fill) and handler (MODE_NAMES)."""
    ms = (ctypes.c_float * (2 * NMODES))()
    ln = (ctypes.c_int64 * (2 * NMODES))()
    _check(lib().slg_kernel_stats(g.handle, 1 if reset else 0, ms, ln))
    return ([list(ms[0:NMODES]), list(ms[NMODES:])], [list(ln[0:NMODES]), list(ln[NMODES:])])


MODE_STATS_COLS = 7
MODE_STATS_NAMES = ("rows", "wedges", "incidences", "pairs", "nonhub_wedges",
                    "scanned_count", "scanned_fill")


def slg_mode_stats(g: Graph, s: int):
    """[[rows, wedges, incidences, pairs, nonhub_wedges, scanned_count, scanned_fill]
    per handler (MODE_NAMES)]; see include/slg.h."""
    c = MODE_STATS_COLS
    out = (ctypes.c_int64 * (c * NMODES))()
    _check(lib().slg_mode_stats(g.handle, s, out))
    return [list(out[c * k:c * k + c]) for k in range(NMODES)]


def slg_ensemble_mode_stats(g: Graph, s_list, which: int):
    """slg_mode_stats for list `which` of the ensemble s_list."""
    a, ap, k = _s_list(s_list)
    c = MODE_STATS_COLS
    out = (ctypes.c_int64 * (c * NMODES))()
    _check(lib().slg_ensemble_mode_stats(g.handle, ap, k, which, out))
    return [list(out[c * q:c * q + c]) for q in range(NMODES)]


def slg_kernel_launches() -> int:
    return int(lib().slg_kernel_launches())


def slg_dual(g: Graph, stream=None) -> Graph:
    """The dual H*; its s-line graphs are the s-clique graphs of H."""
    h = _vp()
    _check(lib().slg_dual(g.handle, _stream_handle(stream), ctypes.byref(h)))
    mm, nn, nz = _i32(), _i32(), _i64()
    _check(lib().slg_graph_info(h, ctypes.byref(mm), ctypes.byref(nn), ctypes.byref(nz)))
    return Graph(h.value, mm.value, nn.value, nz.value)


def slg_batch_load(graphs, s_list, stream=None) -> Graph:
    """One handle over many graphs, each with its own s (pass s=0 to its calls)."""
    k = len(graphs)
    arr = (_vp * k)(*[g.handle for g in graphs])
    s_arr = np.ascontiguousarray(s_list, dtype=np.int32)
    h = _vp()
    _check(lib().slg_batch_load(arr, s_arr.ctypes.data_as(_i32p), k, _stream_handle(stream),
                                ctypes.byref(h)))
    mm, nn, nz = _i32(), _i32(), _i64()
    _check(lib().slg_graph_info(h, ctypes.byref(mm), ctypes.byref(nn), ctypes.byref(nz)))
    return Graph(h.value, mm.value, nn.value, nz.value)


def slg_batch_info(g: Graph) -> np.ndarray:
    """row_base[0..k] of a batch."""
    k = _i32()
    _check(lib().slg_batch_info(g.handle, ctypes.byref(k), None))
    rb = np.zeros(k.value + 1, np.int32)
    _check(lib().slg_batch_info(g.handle, ctypes.byref(k), rb.ctypes.data_as(_i32p)))
    return rb


def slg_batch_pair_offsets(g: Graph) -> np.ndarray:
    """pair_base[0..k] of a batch."""
    k = len(slg_batch_info(g)) - 1
    out = np.zeros(k + 1, np.int64)
    _check(lib().slg_batch_pair_offsets(g.handle, out.ctypes.data_as(_i64p)))
    return out


def slg_batch(graphs, s_list, want_lists=False):
    """s-line graphs of many graphs, each with its own s, in one call.

    Returns one dict per member: pairs, wedges, digest and, when want_lists
    (a bool, or one bool per member), the list as numpy arrays I, J, O
    (member-local ids, canonical order)."""
    k = len(graphs)
    arr = (_vp * k)(*[g.handle for g in graphs])
    s_arr = np.ascontiguousarray(s_list, dtype=np.int32)
    want = [bool(want_lists)] * k if isinstance(want_lists, bool) else [bool(x) for x in want_lists]
    res = (BatchResult * k)()
    for b in range(k):
        res[b].want_list = 1 if want[b] else 0
    _check(lib().slg_batch(arr, s_arr.ctypes.data_as(_i32p), k, res))
    out = []
    for b in range(k):
        r = res[b]
        d = {"status": r.status, "pairs": r.pairs, "wedges": r.wedges, "digest": r.digest}
        if want[b]:
            n = r.pairs
            for name in ("I", "J", "O"):
                p = getattr(r, name)
                d[name] = (np.ctypeslib.as_array(p, shape=(n,)).copy() if n and p
                           else np.zeros(0, np.int32))
            lib().slg_result_free(ctypes.byref(r))
        out.append(d)
    return out


class Server:
    """A query server (handle of libslg's slg_server)."""

    def __init__(self, memory_budget: int, window_pairs: int, max_result_pairs: int,
                 workers: int = 4, max_s: int = 16, digest: bool = True, policy: int = 0,
                 small_workers: int = 0, small_wedges: int = 0, batch_max: int = 0):
        cfg = ServeCfg(memory_budget, window_pairs, max_result_pairs, workers, max_s,
                       1 if digest else 0, policy, small_workers, batch_max, small_wedges)
        h = _vp()
        _check(lib().slg_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h.value
        self._graphs = []

    def close(self):
        if self._h:
            lib().slg_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def slg_serve_create(memory_budget: int, window_pairs: int, max_result_pairs: int,
                     workers: int = 4, max_s: int = 16, digest: bool = True, policy: int = 0,
                     small_workers: int = 0, small_wedges: int = 0,
                     batch_max: int = 0) -> Server:
    return Server(memory_budget, window_pairs, max_result_pairs, workers, max_s, digest, policy,
                  small_workers, small_wedges, batch_max)


def slg_serve_destroy(srv: Server):
    srv.close()


def slg_serve_register(srv: Server, g: Graph) -> int:
    gid = _i32()
    _check(lib().slg_serve_register(srv._h, g.handle, ctypes.byref(gid)))
    srv._graphs.append(g)
    return gid.value


def slg_serve_submit(srv: Server, graph_id: int, s: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().slg_serve_submit(srv._h, graph_id, s, ctypes.byref(t)))
    return t.value


def slg_serve_poll(srv: Server, ticket: int, timeout_ms: int = 60000) -> dict:
    r = ServeResult()
    _check(lib().slg_serve_poll(srv._h, ticket, timeout_ms, ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in ServeResult._fields_}


def slg_serve_fetch(srv: Server, ticket: int, pairs: int):
    I = np.zeros(max(pairs, 1), np.int32)
    J = np.zeros(max(pairs, 1), np.int32)
    O = np.zeros(max(pairs, 1), np.int32)
    _check(lib().slg_serve_fetch(srv._h, ticket, _ptr(I), _ptr(J), _ptr(O), pairs))
    return I[:pairs], J[:pairs], O[:pairs]


def slg_serve_release(srv: Server, ticket: int):
    _check(lib().slg_serve_release(srv._h, ticket))


def slg_serve_stats(srv: Server, reset: bool = False) -> dict:
    st = ServeStats()
    _check(lib().slg_serve_stats(srv._h, 1 if reset else 0, ctypes.byref(st)))
    out = {k: getattr(st, k) for k, _ in ServeStats._fields_}
    if st.batch_failures:
        out["batch_error"] = (lib().slg_last_error() or b"").decode()
    return out


def slg_scan_counts_noalloc(counts, offsets, stream=None):
    """Exclusive scan of int32 device counts into int64 device offsets (n+1).

    Performs no device allocation (see include/slg.h); both tensors must be
    on the GPU.
    """
    n = len(counts)
    _check(lib().slg_scan_counts_noalloc(_ptr(counts), _ptr(offsets), n,
                                         _stream_handle(stream)))
    return offsets


def slg_set_bins(g: Graph, warp_max_wedges: int = 128, block_item_wedges: int = 1024,
                 dense_min_density: int = 64, dense_item_tiles: int = 4,
                 wdense_max_ranges: int = 32, sparse_min_per_tile: int = 64,
                 sparse_item_wedges: int = 65536, wsparse_max_size: int = 32):
    _check(lib().slg_set_bins(g.handle, warp_max_wedges, block_item_wedges, dense_min_density,
                              dense_item_tiles, wdense_max_ranges, sparse_min_per_tile,
                              sparse_item_wedges, wsparse_max_size))


def slg_set_hub_pairs(g: Graph, max_hubs: int = 4096, min_sparse_wedges: int = 1 << 33):
    """Hub-pair handler for sparse rows at s >= 2 (max_hubs = 0 disables it)."""
    _check(lib().slg_set_hub_pairs(g.handle, max_hubs, min_sparse_wedges))


def slg_set_staging(g: Graph, max_bytes: int = -1):
    """The counting pass's staging pool: -1 automatic, 0 off, > 0 at most this many bytes."""
    _check(lib().slg_set_staging(g.handle, max_bytes))


def slg_set_ensemble_filter(g: Graph, mode: int = -1):
    """Lists after the first of an all-list ensemble window: -1 automatic, 0 walk, 1 filter."""
    _check(lib().slg_set_ensemble_filter(g.handle, mode))


def slg_ensemble_fill_stats(g: Graph, reset: bool = False) -> np.ndarray:
    """Per list index of all-list ensemble windows: [windows walked, pairs walked,
    windows filtered, pairs filtered, filter device microseconds while timing,
    pairs the filter read] (shape ENSEMBLE_MAX x 6)."""
    out = np.zeros((ENSEMBLE_MAX, 6), np.int64)
    _check(lib().slg_ensemble_fill_stats(g.handle, int(bool(reset)), out.ctypes.data_as(_i64p)))
    return out


def slg_staging_stats(g: Graph) -> dict:
    """The last counting pass's staging: pool and chunk sizes (pairs), items staged, plan items."""
    out = np.zeros(4, np.int64)
    _check(lib().slg_staging_stats(g.handle, out.ctypes.data_as(_i64p)))
    return {"pool_pairs": int(out[0]), "chunk_pairs": int(out[1]), "items_staged": int(out[2]),
            "items": int(out[3])}


def slg_autotune(g: Graph, s: int, max_trials: int = 24):
    """Pick the binning thresholds for s by timing them on g (kept on g).

    Returns (thresholds in slg_set_bins order, trial time in ms)."""
    bins = np.zeros(8, np.int32)
    ms = ctypes.c_float()
    _check(lib().slg_autotune(g.handle, s, max_trials, bins.ctypes.data_as(_i32p),
                              ctypes.byref(ms)))
    return [int(x) for x in bins], ms.value
