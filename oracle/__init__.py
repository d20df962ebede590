"""CPU oracle for s-line graphs -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU product path never does, and the
two share no code: the oracle is plain C (``slg_oracle.c``) compiled with gcc,
loaded here with ctypes.

Functions follow the definitions of the paper (Liu et al., arXiv 2201.11326):
s-incidence and the s-line graph (Section II-B), the weighted adjacency
L = H^T H (Section II-B), the dual incidence H^T (Section II-A). Every overlap
is a plain sorted-list intersection (the all-pairs / "ijk" order of
Section III-B). See ``slg_oracle.c`` for the row digest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_slg.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_validate.restype = ctypes.c_int
            lib.oracle_validate.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_int32]
            lib.oracle_transpose.restype = None
            lib.oracle_transpose.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                             _i32p, _i32p]
            lib.oracle_rows.restype = None
            lib.oracle_rows.argtypes = [_i32p, _i32p, ctypes.c_int32, _i32p, ctypes.c_int64,
                                        _i32p, ctypes.c_int32, _i64p, _u64p, _i64p,
                                        ctypes.c_int]
            lib.oracle_slg.restype = ctypes.c_int64
            lib.oracle_slg.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                       _i32p, _i32p, ctypes.c_int64]
            lib.oracle_row_list.restype = ctypes.c_int64
            lib.oracle_row_list.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _i32p, _i32p, ctypes.c_int64]
            lib.oracle_list_digest.restype = ctypes.c_uint64
            lib.oracle_list_digest.argtypes = [_i32p, _i32p, _i32p, ctypes.c_int64]
            lib.oracle_slg_fill_rows.restype = None
            lib.oracle_slg_fill_rows.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                                 _i64p, _i32p, _i32p, _i32p, ctypes.c_int]
            lib.oracle_mix.restype = ctypes.c_uint64
            lib.oracle_mix.argtypes = [ctypes.c_uint64]
            lib.oracle_pair_hash.restype = ctypes.c_uint64
            lib.oracle_pair_hash.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int32]
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


def _csr(off, idx):
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, np.int32)  # valid pointer for an empty incidence
    return off, idx


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
               else (os.cpu_count() or 1))


def validate(off, idx, n: int) -> bool:
    """True when every row is a strictly increasing list of ids in [0, n)."""
    off, idx = _csr(off, idx)
    return _load().oracle_validate(_p32(off), _p32(idx), off.size - 1, n) == 0


def transpose(off, idx, n: int):
    """Dual incidence H^T: (offT[n+1], idxT[nnz]) with adj(v) ascending."""
    off, idx = _csr(off, idx)
    m = off.size - 1
    offT = np.zeros(n + 1, np.int32)
    idxT = np.zeros(max(int(off[-1]), 1), np.int32)
    _load().oracle_transpose(_p32(off), _p32(idx), m, n, _p32(offT), _p32(idxT))
    return offT, idxT[:int(off[-1])]


def slg(off, idx, s: int):
    """Full edge list of L_s(H): (I, J, O) int32 arrays sorted by (i, j)."""
    off, idx = _csr(off, idx)
    m = off.size - 1
    lib = _load()
    z = np.zeros(1, np.int32)
    total = lib.oracle_slg(_p32(off), _p32(idx), m, s, _p32(z), _p32(z), _p32(z), 0)
    if total < 0:
        raise ValueError("s must be >= 1")
    I = np.zeros(max(total, 1), np.int32)
    J = np.zeros(max(total, 1), np.int32)
    O = np.zeros(max(total, 1), np.int32)
    lib.oracle_slg(_p32(off), _p32(idx), m, s, _p32(I), _p32(J), _p32(O), total)
    return I[:total], J[:total], O[:total]


def slg_par(off, idx, s: int, nthreads: int | None = None):
    """Same list as ``slg``, rows spread over threads (per-row counts first)."""
    if s < 1:
        raise ValueError("s must be >= 1")
    counts, _, _ = rows(off, idx, None, [s], nthreads)
    off, idx = _csr(off, idx)
    m = off.size - 1
    rowoff = np.zeros(m + 1, np.int64)
    np.cumsum(counts[:, 0], out=rowoff[1:])
    total = int(rowoff[-1])
    I = np.zeros(max(total, 1), np.int32)
    J = np.zeros(max(total, 1), np.int32)
    O = np.zeros(max(total, 1), np.int32)
    if m:
        _load().oracle_slg_fill_rows(_p32(off), _p32(idx), m, s, rowoff.ctypes.data_as(_i64p),
                                     _p32(I), _p32(J), _p32(O), nthreads or default_threads())
    return I[:total], J[:total], O[:total]


def row_list(off, idx, i: int, s: int):
    """Row i of L_s(H): (J, O) for all j > i with overlap >= s, ascending j."""
    off, idx = _csr(off, idx)
    m = off.size - 1
    cap = max(m - i - 1, 1)
    J = np.zeros(cap, np.int32)
    O = np.zeros(cap, np.int32)
    c = _load().oracle_row_list(_p32(off), _p32(idx), m, i, s, _p32(J), _p32(O), cap)
    return J[:c], O[:c]


def rows(off, idx, row_ids, s_list, nthreads: int | None = None):
    """Per-row (count, digest, overlap_sum) arrays of shape [len(rows), len(s_list)].

    ``row_ids=None`` evaluates every row. overlap_sum is the sum of
    |e_i ∩ e_j| over j > i with |e_i|, |e_j| >= s.
    """
    off, idx = _csr(off, idx)
    m = off.size - 1
    s_arr = np.ascontiguousarray(np.atleast_1d(s_list), dtype=np.int32)
    if row_ids is None:
        r = None
        nr = m
        rp = ctypes.cast(None, _i32p)
    else:
        r = np.ascontiguousarray(row_ids, dtype=np.int32)
        nr = r.size
        rp = _p32(r) if nr else ctypes.cast(None, _i32p)
    counts = np.zeros((max(nr, 1), s_arr.size), np.int64)
    digests = np.zeros((max(nr, 1), s_arr.size), np.uint64)
    osum = np.zeros((max(nr, 1), s_arr.size), np.int64)
    if nr:
        _load().oracle_rows(_p32(off), _p32(idx), m, rp, nr, _p32(s_arr), s_arr.size,
                            counts.ctypes.data_as(_i64p), digests.ctypes.data_as(_u64p),
                            osum.ctypes.data_as(_i64p), nthreads or default_threads())
    return counts[:nr], digests[:nr], osum[:nr]


def list_digest(I, J, O) -> int:
    """Digest of an explicit list (rows contiguous), same definition as ``rows``."""
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    O = np.ascontiguousarray(O, dtype=np.int32)
    if I.size == 0:
        return 0
    return int(_load().oracle_list_digest(_p32(I), _p32(J), _p32(O), I.size))


def mix(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014) of a 64-bit word."""
    return int(_load().oracle_mix(x % 2**64))


def pair_hash(i: int, k: int, j: int, o: int) -> int:
    return int(_load().oracle_pair_hash(i, k, j, o))
