"""Seeded synthetic hypergraphs shaped like the paper's workloads (Section VI, dataset table).

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark. It holds no s-line arithmetic: it only draws hyperedge sizes and
member vertices and returns a hypergraph as int32 CSR incidence
(``off[m+1]``, ``idx[nnz]``; row i lists the vertices of hyperedge e_i in
ascending order).

Recipe (every draw comes from numpy's PCG64 via ``default_rng``):

* sizes: "Zipf(a) clipped [lo, hi]" is ``clip(zipf(a), lo, hi)``;
  "log-normal(mu, sigma) clipped [lo, hi]" is ``clip(rint(exp(N(mu, sigma))), lo, hi)``.
  Clipping clamps, it never redraws.
* popularity: "Zipf(a)" gives the vertex of popularity rank r (1-based) the
  weight r^-a; ranks are mapped to vertex ids by a seeded permutation.
  "Chung-Lu Zipf(a) capped at c" draws a target degree ``clip(zipf(a), 1, c)``
  per vertex and uses it as the weight.
* members: each hyperedge takes the first |e| distinct vertices of an i.i.d.
  weighted draw sequence (sequential weighted sampling without replacement,
  i.e. rejection of repeats), then the row is sorted.
* streams: sizes come from ``default_rng([*seed, 0])``, the popularity
  permutation / target degrees from ``default_rng([*seed, 1])`` and the
  members of row chunk c (rows ``[c*2**18, (c+1)*2**18)``) from
  ``default_rng([*seed, 2, c])``, so a chunk can be drawn without the others.
* the batched, served and large workloads draw members with the same rule in
  C (``fastgen.c``: alias-method draws, rejection of repeats, threaded over
  rows, row r on the SplitMix64 stream keyed by the seed and r); their sizes
  and popularity still come from the numpy streams above.

A hyperedge size is clamped to n so that every row can be filled.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile
import threading
from typing import Sequence

import numpy as np

CHUNK_ROWS = 1 << 18


@dataclasses.dataclass(frozen=True)
class Hypergraph:
    """Hyperedge -> vertex incidence in CSR form (int32)."""

    off: np.ndarray  # int32 [m+1]
    idx: np.ndarray  # int32 [nnz]
    n: int
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.off.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.idx.size)

    def row(self, i: int) -> np.ndarray:
        return self.idx[self.off[i]:self.off[i + 1]]

    def sizes(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)


# ----------------------------------------------------------------------------
# size distributions
# ----------------------------------------------------------------------------

def sizes_zipf(rng: np.random.Generator, m: int, a: float, lo: int, hi: int) -> np.ndarray:
    return np.clip(rng.zipf(a, size=m), lo, hi).astype(np.int64)


def sizes_lognormal(rng: np.random.Generator, m: int, mu: float, sigma: float,
                    lo: int, hi: int) -> np.ndarray:
    x = np.rint(np.exp(rng.normal(mu, sigma, size=m)))
    return np.clip(x, lo, hi).astype(np.int64)


# ----------------------------------------------------------------------------
# popularity (weights per vertex id)
# ----------------------------------------------------------------------------

def popularity_zipf(rng: np.random.Generator, n: int, a: float) -> np.ndarray:
    ranks = np.arange(1, n + 1, dtype=np.float64)
    w_by_rank = ranks ** (-a)
    perm = rng.permutation(n)          # perm[r] = vertex id of rank r+1
    w = np.empty(n, np.float64)
    w[perm] = w_by_rank
    return w


def popularity_chung_lu(rng: np.random.Generator, n: int, a: float, cap: int) -> np.ndarray:
    return np.clip(rng.zipf(a, size=n), 1, cap).astype(np.float64)


# ----------------------------------------------------------------------------
# members: sequential weighted sampling without replacement
# ----------------------------------------------------------------------------

def _draw_chunk(rng: np.random.Generator, sizes: np.ndarray, order: np.ndarray,
                cdf: np.ndarray) -> np.ndarray:
    """Members for one chunk of rows, concatenated in row order, rows sorted.

    ``order`` lists vertex ids by decreasing weight and ``cdf`` is the
    cumulative weight along that order (last entry 1.0).
    """
    n = order.size
    m = sizes.size
    off = np.zeros(m + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    out = np.empty(int(off[-1]), np.int64)
    have = np.zeros(m, np.int64)
    active = np.flatnonzero(sizes > 0)
    mult = 2
    while active.size:
        need = sizes[active] - have[active]
        b = np.minimum(need * mult + 4, 1 << 16)
        rows = np.repeat(active, b)
        pos = np.searchsorted(cdf, rng.random(int(b.sum())), side="right")
        cand = order[np.minimum(pos, n - 1)]
        # already accepted members of the active rows go first so that they win
        # the first-occurrence test below
        have_a = have[active]
        old_rows = np.repeat(active, have_a)
        starts = np.repeat(off[active], have_a)
        within = np.arange(old_rows.size, dtype=np.int64) - np.repeat(
            np.cumsum(have_a) - have_a, have_a)
        old_vals = out[starts + within]
        keys = np.concatenate([old_rows * n + old_vals, rows * n + cand])
        _, first = np.unique(keys, return_index=True)   # first occurrence (stable)
        first = np.sort(first[first >= old_rows.size]) - old_rows.size
        r = rows[first]
        # rank of each new distinct value within its row, in draw order
        grp_start = np.flatnonzero(np.r_[True, r[1:] != r[:-1]])
        counts = np.diff(np.r_[grp_start, r.size])
        rank = np.arange(r.size) - np.repeat(grp_start, counts)
        take = rank < (sizes[r] - have[r])
        r_t = r[take]
        out[off[r_t] + have[r_t] + rank[take]] = cand[first[take]]
        np.add.at(have, r_t, 1)
        active = active[have[active] < sizes[active]]
        mult = min(mult * 2, 64)
    row_id = np.repeat(np.arange(m, dtype=np.int64), sizes)
    out = out[np.lexsort((out, row_id))]
    return out


def members(seed: Sequence[int], sizes: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """Concatenated sorted rows (int64) for the given sizes and vertex weights."""
    n = weights.size
    order = np.argsort(-weights, kind="stable")
    cdf = np.cumsum(weights[order])
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    parts = []
    m = sizes.size
    for c, r0 in enumerate(range(0, m, CHUNK_ROWS)):
        rng = np.random.default_rng([*seed, 2, c])
        parts.append(_draw_chunk(rng, sizes[r0:r0 + CHUNK_ROWS], order, cdf))
    return np.concatenate(parts) if parts else np.zeros(0, np.int64)


_HERE = os.path.dirname(os.path.abspath(__file__))
_FG_SRC = os.path.join(_HERE, "fastgen.c")
_FG_LIB = os.path.join(_HERE, "_build", "libfastgen.so")
_fg_lock = threading.Lock()
_fg = None


def build_fastgen(force: bool = False) -> str:
    """Compile the C member draw (plain gcc -O2)."""
    os.makedirs(os.path.dirname(_FG_LIB), exist_ok=True)
    if force or not os.path.exists(_FG_LIB) or (
            os.path.getmtime(_FG_LIB) < os.path.getmtime(_FG_SRC)):
        tmp = _FG_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o",
                               tmp, _FG_SRC, "-lm"])
        os.replace(tmp, _FG_LIB)
    return _FG_LIB


def _fastgen():
    global _fg
    with _fg_lock:
        if _fg is None:
            lib = ctypes.CDLL(build_fastgen())
            lib.fastgen_members.restype = ctypes.c_int
            lib.fastgen_members.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_int]
            _fg = lib
    return _fg


def members_fast(seed: Sequence[int], sizes: np.ndarray, weights: np.ndarray):
    """Same rule as ``members``, drawn in C; returns (off int64 [m+1], idx int32)."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    off = np.zeros(sizes.size + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = np.empty(max(int(off[-1]), 1), np.int32)
    key = int(np.random.SeedSequence([*seed, 3]).generate_state(1, dtype=np.uint64)[0])
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4
    rc = _fastgen().fastgen_members(sizes.size, sizes.ctypes.data, off.ctypes.data,
                                    w.ctypes.data, w.size, key, idx.ctypes.data, threads)
    if rc != 0:
        raise MemoryError("fastgen_members failed")
    return off, idx[:int(off[-1])]


def build(seed: Sequence[int], m: int, n: int, size_kind: str, size_args: tuple,
          pop_kind: str, pop_args: tuple, name: str = "", fast: bool = False) -> Hypergraph:
    seed = tuple(int(x) for x in seed)
    rs = np.random.default_rng([*seed, 0])
    if size_kind == "zipf":
        sizes = sizes_zipf(rs, m, *size_args)
    elif size_kind == "lognormal":
        sizes = sizes_lognormal(rs, m, *size_args)
    else:
        raise ValueError(size_kind)
    sizes = np.minimum(sizes, n)
    rp = np.random.default_rng([*seed, 1])
    if pop_kind == "zipf":
        w = popularity_zipf(rp, n, *pop_args)
    elif pop_kind == "chung_lu":
        w = popularity_chung_lu(rp, n, *pop_args)
    else:
        raise ValueError(pop_kind)
    if fast:
        off, idx = members_fast(seed, sizes, w)
    else:
        idx = members(seed, sizes, w)
        off = np.zeros(m + 1, np.int64)
        np.cumsum(sizes, out=off[1:])
    if off[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 offsets")
    return Hypergraph(off.astype(np.int32), idx.astype(np.int32), int(n), name)


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def tiny(seed: int = 0) -> Hypergraph:
    """m=2,000 over n=1,000; sizes Zipf(2.1) clipped [2,100]; popularity Zipf(1.5)."""
    return build((seed,), 2000, 1000, "zipf", (2.1, 2, 100), "zipf", (1.5,), "tiny")


def medium(seed: int = 0, m: int = 1_000_000, n: int | None = None) -> Hypergraph:
    """m=1M over n=500k; sizes log-normal(1.8, 1.0) clipped [2,5000]; popularity Zipf(1.7).

    ``m`` (and ``n``, default m/2) scale the same recipe down for parity cases.
    """
    n = m // 2 if n is None else n
    return build((seed,), m, n, "lognormal", (1.8, 1.0, 2, 5000), "zipf", (1.7,),
                 f"medium_m{m}")


def large(seed: int = 0, m: int = 20_000_000, n: int | None = None) -> Hypergraph:
    """m=20M over n=10M; sizes log-normal(2.0, 1.1) clipped [2,20000];
    Chung-Lu popularity with vertex degree Zipf(1.8) capped at 100,000."""
    n = m // 2 if n is None else n
    return build((seed,), m, n, "lognormal", (2.0, 1.1, 2, 20000), "chung_lu",
                 (1.8, 100_000), f"large_m{m}", fast=True)


def batch_member(b: int, base_seed: int = 0) -> tuple[Hypergraph, int]:
    """Graph b of the batched workload and its s.

    m is log-uniform in [100, 100000], n = m/2, sizes and popularity as in
    ``medium``; s is uniform in {1,2,3,4}. Graph b uses seed (base_seed, b).
    """
    rng = np.random.default_rng([base_seed, b, 9])
    m = int(np.rint(np.exp(rng.uniform(np.log(100), np.log(100_000)))))
    s = int(rng.integers(1, 5))
    g = build((base_seed, b), m, max(m // 2, 1), "lognormal", (1.8, 1.0, 2, 5000), "zipf",
              (1.7,), f"batch{b}_m{m}", fast=True)
    return g, s


def served_member(g: int, base_seed: int = 0) -> Hypergraph:
    """Resident graph g of the served workload: g < 8 are medium-sized
    (m=1M), the others have m log-uniform in [1e3, 1e5]."""
    if g < 8:
        m = 1_000_000
    else:
        rng = np.random.default_rng([base_seed, 1000 + g, 9])
        m = int(np.rint(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
    return build((base_seed, 1000 + g), m, m // 2, "lognormal", (1.8, 1.0, 2, 5000), "zipf",
                 (1.7,), f"served{g}_m{m}", fast=True)


def uniform_random(seed: int, m: int, n: int, lo: int, hi: int) -> Hypergraph:
    """Small hypergraphs for brute-force checks: sizes uniform in [lo, hi],
    members uniform without replacement."""
    rng = np.random.default_rng([seed, 77])
    sizes = np.minimum(rng.integers(lo, hi + 1, size=m), n)
    rows = [np.sort(rng.choice(n, size=int(k), replace=False)) for k in sizes]
    off = np.zeros(m + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    return Hypergraph(off.astype(np.int32), idx.astype(np.int32), int(n), f"uniform{seed}")


def striped_hub(seed: int, m: int, n: int, period: int, lo: int = 1, hi: int = 4) -> Hypergraph:
    """A sparse graph whose hub rows span many j tiles.

    Every row draws a uniform size in [lo, hi] of distinct vertices from
    [1, n); rows i with i % period == 0 also contain vertex 0, so the hub list
    adj(0) covers the whole id range with density 1/period.
    """
    rng = np.random.default_rng([seed, 78])
    sizes = rng.integers(lo, hi + 1, size=m)
    rows = []
    for i, k in enumerate(sizes):
        r = rng.choice(np.arange(1, n), size=int(min(k, n - 1)), replace=False)
        if i % period == 0:
            r = np.append(r, 0)
        rows.append(np.sort(r))
    off = np.zeros(m + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=off[1:])
    idx = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    return Hypergraph(off.astype(np.int32), idx.astype(np.int32), int(n), f"striped{seed}")


# ----------------------------------------------------------------------------
# file cache (int32 CSR binaries)
# ----------------------------------------------------------------------------

def cache_dir() -> str:
    d = os.environ.get("SLG_SYNTH_CACHE") or os.path.join(tempfile.gettempdir(), "slg_synth")
    os.makedirs(d, exist_ok=True)
    return d


def save(h: Hypergraph, path: str) -> None:
    # a temporary file per process, renamed into place: processes that build the
    # same graph at once (ranks on one host) never read a partial file
    hdr = np.array([h.m, h.n, h.nnz], np.int64)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as f:
        hdr.tofile(f)
        h.off.astype(np.int32).tofile(f)
        h.idx.astype(np.int32).tofile(f)
    os.replace(tmp, path)


def load(path: str, name: str = "") -> Hypergraph:
    with open(path, "rb") as f:
        m, n, nnz = (int(x) for x in np.fromfile(f, np.int64, 3))
        off = np.fromfile(f, np.int32, m + 1)
        idx = np.fromfile(f, np.int32, nnz)
    return Hypergraph(off, idx, n, name)


def cached(key: str, make) -> Hypergraph:
    path = os.path.join(cache_dir(), key + ".csr")
    if os.path.exists(path):
        return load(path, key)
    h = make()
    save(h, path)
    return h
