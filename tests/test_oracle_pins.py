"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test ties the oracle to the paper's worked example, to a different
algorithm (bitset popcount, a scipy sparse H^T H), to a closed form, or to an
identity of the definitions, so that a dropped term, a wrong comparison, an
off-by-one in j or a transposed operand in the oracle fails at least one of
them. No GPU is needed.
"""
from math import comb
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

# ---------------------------------------------------------------- helpers


def csr_from_rows(rows):
    off = np.zeros(len(rows) + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in rows])
    idx = np.array([v for r in rows for v in sorted(r)], np.int32)
    return off, idx


def parse_golden(path):
    edges, pairs, es, adj, inc = {}, {}, {}, [], []
    n = None
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            k, vals = tok[0], [int(x) for x in tok[1:]]
            if k == "n":
                n = vals[0]
            elif k == "edge":
                edges[vals[0]] = vals[1:]
            elif k == "pair":
                pairs.setdefault(vals[0], []).append(tuple(vals[1:]))
            elif k == "Es":
                es[vals[0]] = vals[1:]
            elif k == "adj":
                adj.append(vals)
            elif k == "inc":
                inc.append(vals)
    rows = [edges[i] for i in range(len(edges))]
    return n, rows, pairs, es, adj, inc


def bitset_pairs(rows, s):
    """All-pairs overlaps by popcount of vertex bitmasks (a different algorithm)."""
    masks = [sum(1 << v for v in r) for r in rows]
    out = []
    for i in range(len(rows)):
        for j in range(i + 1, len(rows)):
            o = bin(masks[i] & masks[j]).count("1")
            if o >= s:
                out.append((i, j, o))
    return out


def as_triples(I, J, O):
    return list(zip(I.tolist(), J.tolist(), O.tolist()))


def sparse_upper(off, idx, n, s):
    """Strict upper triangle of H^T H thresholded at s (scipy SpGEMM)."""
    m = off.size - 1
    H = sp.csr_matrix((np.ones(idx.size, np.int64), idx, off), shape=(m, n))  # rows = e_i
    L = (H @ H.T).tocoo()  # m x m, L[i,j] = |e_i ∩ e_j|
    keep = (L.row < L.col) & (L.data >= s)
    t = sorted(zip(L.row[keep].tolist(), L.col[keep].tolist(), L.data[keep].tolist()))
    return t


def wedges_by_definition(off, idx, n, s):
    """W_{s,i} = sum over v in e_i of #{j > i : v in e_j, |e_j| >= s}, for |e_i| >= s.

    Computed from vertex degrees restricted to E_s, without any overlap.
    """
    m = off.size - 1
    sizes = np.diff(off)
    row = np.repeat(np.arange(m), sizes)
    keep = sizes[row] >= s
    per_row = np.zeros(m, np.int64)
    # for each vertex, the kept rows containing it, ascending; an entry at
    # position p of a list of length d has d-1-p later entries
    v = idx[keep]
    r = row[keep]
    order = np.lexsort((r, v))
    v_sorted, r_sorted = v[order], r[order]
    starts = np.searchsorted(v_sorted, v_sorted, side="left")
    ends = np.searchsorted(v_sorted, v_sorted, side="right")
    pos = np.arange(v_sorted.size) - starts
    later = ends - starts - 1 - pos
    np.add.at(per_row, r_sorted, later)
    ds = np.bincount(v, minlength=n).astype(np.int64)
    total = int((ds * (ds - 1) // 2).sum())
    return per_row, total


# ---------------------------------------------------------- worked example


def test_worked_example(golden_dir):
    n, rows, pairs, es, adj_facts, inc_facts = parse_golden(
        os.path.join(golden_dir, "worked_example.txt"))
    off, idx = csr_from_rows(rows)
    assert oracle.validate(off, idx, n)
    for s in range(1, 6):
        got = as_triples(*oracle.slg(off, idx, s))
        assert got == sorted(pairs.get(s, [])), s
    # E_s from sizes (Section II-B)
    sizes = np.diff(off)
    for s, ids in es.items():
        assert np.flatnonzero(sizes >= s).tolist() == ids
    # adj(u,v) = number of hyperedges containing both u and v, through the dual
    offT, idxT = oracle.transpose(off, idx, n)
    for u, v, val in adj_facts:
        au = set(idxT[offT[u]:offT[u + 1]].tolist())
        av = set(idxT[offT[v]:offT[v + 1]].tolist())
        assert len(au & av) == val
    for vals in inc_facts:
        ids, val = vals[:-1], vals[-1]
        common = set(rows[ids[0]])
        for e in ids[1:]:
            common &= set(rows[e])
        assert len(common) == val


def test_worked_example_dual():
    # H* of the example: adj(v) ascending, vertices a..f
    rows = [[0, 1, 2], [1, 2, 3], [0, 1, 2, 3, 4], [4, 5]]
    off, idx = csr_from_rows(rows)
    offT, idxT = oracle.transpose(off, idx, 6)
    adj = [idxT[offT[v]:offT[v + 1]].tolist() for v in range(6)]
    assert adj == [[0, 2], [0, 1, 2], [0, 1, 2], [1, 2], [2, 3], [3]]


# ----------------------------------------------------------- brute force


@pytest.mark.parametrize("seed", range(12))
def test_bitset_bruteforce(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 65))
    n = int(rng.integers(1, 129))
    h = synth.uniform_random(seed, m, n, 0, min(n, 12))
    rows = [h.row(i).tolist() for i in range(m)]
    for s in (1, 2, 3, 5):
        assert as_triples(*oracle.slg(h.off, h.idx, s)) == bitset_pairs(rows, s)


@pytest.mark.parametrize("seed", range(4))
def test_row_api_matches_full_list(seed):
    h = synth.uniform_random(100 + seed, 60, 40, 1, 15)
    rows = [h.row(i).tolist() for i in range(h.m)]
    for s in (1, 2, 4):
        ref = bitset_pairs(rows, s)
        for i in range(h.m):
            J, O = oracle.row_list(h.off, h.idx, i, s)
            assert list(zip([i] * J.size, J.tolist(), O.tolist())) == [t for t in ref if t[0] == i]
        counts, dig, _ = oracle.rows(h.off, h.idx, None, [s])
        per_row = np.bincount([t[0] for t in ref], minlength=h.m) if ref else np.zeros(h.m)
        assert counts[:, 0].tolist() == per_row.tolist()


# -------------------------------------------------- library cross-checks


def test_tiny_workload_vs_scipy_spgemm():
    h = synth.tiny()
    for s in (1, 2, 3):
        got = as_triples(*oracle.slg(h.off, h.idx, s))
        assert got == sparse_upper(h.off, h.idx, h.n, s)
        assert len(got) > 0


@pytest.mark.parametrize("seed", range(3))
def test_medium_recipe_small_vs_scipy(seed):
    h = synth.medium(seed=seed, m=3000)
    for s in (1, 4, 8):
        assert as_triples(*oracle.slg(h.off, h.idx, s)) == sparse_upper(h.off, h.idx, h.n, s)


def test_threaded_list_equals_single_thread():
    h = synth.medium(seed=9, m=2500)
    for s in (1, 3, 6):
        a = oracle.slg(h.off, h.idx, s)
        b = oracle.slg_par(h.off, h.idx, s, nthreads=3)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    e = synth.uniform_random(5, 0, 10, 0, 3)
    assert oracle.slg_par(e.off, e.idx, 1)[0].size == 0


def test_transpose_vs_scipy():
    h = synth.medium(seed=5, m=5000)
    offT, idxT = oracle.transpose(h.off, h.idx, h.n)
    H = sp.csr_matrix((np.ones(h.nnz), h.idx, h.off), shape=(h.m, h.n)).T.tocsr()
    H.sort_indices()
    assert np.array_equal(offT, H.indptr.astype(np.int32))
    assert np.array_equal(idxT, H.indices.astype(np.int32))


def test_s_clique_is_line_graph_of_dual():
    # Section III-H: W = H H^T - D_V; the s-clique graph joins u, v with
    # W[u, v] >= s, and equals the s-line graph of the dual H*
    h = synth.medium(seed=14, m=1500)
    H = sp.csr_matrix((np.ones(h.nnz, np.int64), h.idx, h.off), shape=(h.m, h.n))
    Wm = (H.T @ H).tocoo()  # n x n: W[u,v] = hyperedges holding both u and v (+ D_V)
    offT, idxT = oracle.transpose(h.off, h.idx, h.n)
    for s in (1, 2, 5):
        keep = (Wm.row < Wm.col) & (Wm.data >= s)
        want = sorted(zip(Wm.row[keep].tolist(), Wm.col[keep].tolist(), Wm.data[keep].tolist()))
        assert as_triples(*oracle.slg(offT, idxT, s)) == want


# ------------------------------------------------------------ closed forms


def test_two_uniform_line_graph_count():
    # s = 1 on a simple graph: |L_1| = sum_v C(deg v, 2) (edges of its line graph)
    rng = np.random.default_rng(7)
    n = 60
    all_pairs = [(u, v) for u in range(n) for v in range(u + 1, n)]
    pick = rng.choice(len(all_pairs), size=300, replace=False)
    rows = [list(all_pairs[k]) for k in pick]
    off, idx = csr_from_rows(rows)
    deg = np.bincount(idx, minlength=n)
    I, J, O = oracle.slg(off, idx, 1)
    assert I.size == int(sum(comb(int(d), 2) for d in deg))
    assert set(O.tolist()) == {1}
    assert oracle.slg(off, idx, 2)[0].size == 0


@pytest.mark.parametrize("q,k", [(7, 3), (8, 4), (9, 4)])
def test_johnson_scheme(q, k):
    # all k-subsets of [q]: pairs at overlap t number C(q,k) C(k,t) C(q-k,k-t) / 2
    rows = [list(c) for c in itertools.combinations(range(q), k)]
    off, idx = csr_from_rows(rows)
    I, J, O = oracle.slg(off, idx, 1)
    hist = np.bincount(O, minlength=k + 1)
    for t in range(1, k):
        assert hist[t] == comb(q, k) * comb(k, t) * comb(q - k, k - t) // 2, t
    assert hist[k] == 0
    for s in range(1, k + 1):
        expect = sum(comb(q, k) * comb(k, t) * comb(q - k, k - t) // 2 for t in range(s, k))
        assert oracle.slg(off, idx, s)[0].size == expect


@pytest.mark.parametrize("p,c", [(5, 2), (9, 4), (12, 1)])
def test_sunflower(p, c):
    core = list(range(c))
    rows, nxt = [], c
    for q in range(p):
        petal = list(range(nxt, nxt + q % 3 + 1))
        nxt += len(petal)
        rows.append(core + petal)
    off, idx = csr_from_rows(rows)
    I, J, O = oracle.slg(off, idx, 1)
    assert I.size == comb(p, 2) and set(O.tolist()) == {c}
    assert oracle.slg(off, idx, c)[0].size == comb(p, 2)
    assert oracle.slg(off, idx, c + 1)[0].size == 0


def test_identical_copies():
    # an indexable family: k copies of one t-set pair with overlap t
    k, t = 6, 5
    rows = [list(range(10, 10 + t))] * k
    off, idx = csr_from_rows(rows)
    I, J, O = oracle.slg(off, idx, t)
    assert I.size == comb(k, 2) and set(O.tolist()) == {t}
    assert as_triples(I, J, O) == [(i, j, t) for i in range(k) for j in range(i + 1, k)]


# ------------------------------------------------------------- invariants


@pytest.mark.parametrize("seed", range(3))
def test_nesting_and_bounds(seed):
    h = synth.medium(seed=seed, m=2000)
    sizes = np.diff(h.off)
    prev = None
    for s in range(1, 9):
        I, J, O = oracle.slg(h.off, h.idx, s)
        assert np.all(I < J)
        key = I.astype(np.int64) * h.m + J
        assert np.all(np.diff(key) > 0)  # sorted by (i, j), no repeats
        assert np.all(O >= s)
        assert np.all(O <= np.minimum(sizes[I], sizes[J]))
        if prev is not None:
            # L_{s} is L_{s-1} restricted to overlap >= s, with the same overlaps
            pI, pJ, pO = prev
            sel = pO >= s
            assert np.array_equal(pI[sel], I) and np.array_equal(pJ[sel], J)
            assert np.array_equal(pO[sel], O)
        prev = (I, J, O)


@pytest.mark.parametrize("seed", range(3))
def test_overlap_sum_equals_wedges(seed):
    # double counting: sum_{j>i} |e_i ∩ e_j| over E_s equals the wedge count W_{s,i},
    # and over all rows sum_v C(d_s(v), 2)
    h = synth.medium(seed=10 + seed, m=3000)
    s_list = [1, 2, 3, 5, 8]
    _, _, osum = oracle.rows(h.off, h.idx, None, s_list)
    for t, s in enumerate(s_list):
        per_row, total = wedges_by_definition(h.off, h.idx, h.n, s)
        assert np.array_equal(osum[:, t], per_row)
        assert int(osum[:, t].sum()) == total


def test_s1_is_intersection_graph():
    # L_1 joins exactly the hyperedges that share a vertex
    h = synth.uniform_random(3, 80, 50, 1, 6)
    I, J, O = oracle.slg(h.off, h.idx, 1)
    got = set(zip(I.tolist(), J.tolist()))
    rows = [set(h.row(i).tolist()) for i in range(h.m)]
    want = {(i, j) for i in range(h.m) for j in range(i + 1, h.m) if rows[i] & rows[j]}
    assert got == want


# ----------------------------------------------------------------- digest


def test_splitmix64_published_vectors():
    # SplitMix64 seeded with 1234567: the k-th output is mix(1234567 + k*gamma);
    # the first five are the published reference values.
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    gamma = 0x9E3779B97F4A7C15
    assert [oracle.mix(1234567 + k * gamma) for k in range(5)] == expected
    # the pair hash nests it: mix(mix((i<<32)|k) ^ ((j<<32)|o))
    for i, k, j, o in [(0, 0, 0, 0), (3, 7, 11, 2), (2**31 - 1, 5, 2**31 - 2, 9)]:
        assert oracle.pair_hash(i, k, j, o) == oracle.mix(
            oracle.mix((i << 32) | k) ^ ((j << 32) | o))


def test_digest_sum_of_rows():
    h = synth.tiny()
    for s in (1, 2, 3):
        I, J, O = oracle.slg(h.off, h.idx, s)
        _, dig, _ = oracle.rows(h.off, h.idx, None, [s])
        total = int(dig[:, 0].astype(np.uint64).sum(dtype=np.uint64))
        assert total == oracle.list_digest(I, J, O)
        # order-sensitive within a row: swapping two entries of one row changes it
        if I.size >= 2 and I[0] == I[1]:
            J2, O2 = J.copy(), O.copy()
            J2[[0, 1]] = J2[[1, 0]]
            O2[[0, 1]] = O2[[1, 0]]
            assert oracle.list_digest(I, J2, O2) != total


# ------------------------------------------------------------- validation


def test_validation_rules():
    ok = csr_from_rows([[0, 2], [1], [], [0, 1, 3]])
    assert oracle.validate(*ok, 4)
    assert not oracle.validate(*ok, 3)  # id 3 out of range
    assert not oracle.validate(np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 2], np.int32), 4)
    assert not oracle.validate(np.array([0, 2, 4], np.int32), np.array([2, 1, 0, 2], np.int32), 4)
    assert not oracle.validate(np.array([0, 3, 2], np.int32), np.array([0, 1, 2], np.int32), 4)
    assert not oracle.validate(np.array([1, 3], np.int32), np.array([0, 1, 2], np.int32), 4)
    assert not oracle.validate(np.array([0, 1], np.int32), np.array([-1], np.int32), 4)


def test_empty_rows_and_large_s():
    off, idx = csr_from_rows([[], [0, 1], [], [0, 1], []])
    assert as_triples(*oracle.slg(off, idx, 1)) == [(1, 3, 2)]
    assert as_triples(*oracle.slg(off, idx, 3)) == []
    off0 = np.zeros(1, np.int32)
    assert oracle.slg(off0, np.zeros(0, np.int32), 1)[0].size == 0
