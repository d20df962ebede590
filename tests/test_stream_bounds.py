"""The bounds one-walk windows choose their rows by (CPU, against the oracle).

A window's rows are picked before they are walked, from an upper bound on each
row's pairs: W_i / s for a row walked through its wedges (a pair with overlap
>= s takes s of the row's wedges to later rows) and E_i / (s - 1) for a row
walked through non-hub wedges and hub-pair lists (a partner sharing u non-hub
vertices and t hubs, u + t >= s >= 2, is met u + t(t-1)/2 times). If either
bound were wrong a window could overflow its buffer; the library would then cut
it, but the bound itself must hold. Both are checked here against the oracle's
per-row counts, and the second by brute force over the hub split of every pair.
"""
import numpy as np
import pytest

import oracle
import synth


def later_wedges(h, s):
    """W_{s,i}: wedges of row i to later rows, both of size >= s."""
    sizes = np.diff(h.off)
    keep = sizes >= s
    W = np.zeros(h.m, np.int64)
    for v_rows in vertex_rows(h):
        r = v_rows[keep[v_rows]]
        # row r[k] meets the len(r) - 1 - k later rows of adj_s(v)
        W[r] += np.arange(r.size - 1, -1, -1)
    return W


def vertex_rows(h):
    offT, idxT = oracle.transpose(h.off, h.idx, h.n)
    return [idxT[offT[v]:offT[v + 1]] for v in range(h.n)]


@pytest.mark.parametrize("seed,m,n,lo,hi", [(1, 300, 60, 2, 12), (2, 500, 40, 3, 20),
                                           (3, 200, 400, 2, 40)])
def test_row_pairs_at_most_wedges_over_s(seed, m, n, lo, hi):
    h = synth.uniform_random(seed, m, n, lo, hi)
    s_list = [1, 2, 3, 5]
    counts, _, osum = oracle.rows(h.off, h.idx, None, s_list)
    for k, s in enumerate(s_list):
        W = later_wedges(h, s)
        # the overlaps with every later row of size >= s add up to the wedges ...
        assert np.array_equal(osum[:, k], W), s
        # ... so the pairs, each of overlap >= s, are at most W / s
        assert np.all(counts[:, k] * s <= W), s


def test_hub_pair_entries_bound_by_brute_force():
    # every split of an overlap u + t >= s into u non-hub and t hub vertices is
    # met at least s - 1 times (u wedges plus one hit per pair of shared hubs)
    for s in range(2, 40):
        worst = min(u + t * (t - 1) // 2
                    for t in range(0, 60) for u in range(0, 60) if u + t >= s)
        assert worst == s - 1, s


def test_hub_pair_entries_bound_on_rows():
    # with a hub set, the entries a row's walk meets (non-hub wedges plus hub
    # pairs in common with each later row) bound its pairs times (s - 1)
    h = synth.uniform_random(4, 400, 50, 3, 25)
    deg = np.bincount(h.idx, minlength=h.n)
    hubs = set(np.argsort(-deg, kind="stable")[:12].tolist())
    rows = [set(h.idx[h.off[i]:h.off[i + 1]].tolist()) for i in range(h.m)]
    for s in (2, 3, 4, 6):
        sizes = np.diff(h.off)
        for i in range(0, h.m, 7):
            if sizes[i] < s:
                continue
            entries = pairs = 0
            for j in range(i + 1, h.m):
                if sizes[j] < s:
                    continue
                common = rows[i] & rows[j]
                t = len(common & hubs)
                u = len(common) - t
                entries += u + t * (t - 1) // 2
                pairs += len(common) >= s
            assert pairs * (s - 1) <= entries, (s, i)
            J, _ = oracle.row_list(h.off, h.idx, i, s)
            assert J.size == pairs
