"""Full-size parity on the medium workload, in the benchmark's launch configuration.

The medium hypergraph (m = 1,000,000) is built through windows of at most 2^33
pairs into reused device buffers, exactly as bench.py times it. Its s-line
graphs hold up to 4.8e11 pairs, so the comparison with the oracle is per row:
for 1,000 seeded random rows and the 100 rows with the most wedges, the
library's per-row pair count and per-row digest (a position-sensitive hash of
the row's list) must equal the oracle's. Globally, the row counts must add up
to |L_s| and, at s = 1, the overlaps of all pairs must add up to
sum_v C(deg v, 2), the closed form of the wedge count.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg

pytestmark = pytest.mark.gpu

WINDOW = 1 << 33


@pytest.fixture(scope="module")
def medium():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    h = synth.cached("medium_m1000000_seed0", lambda: synth.medium(seed=0, m=1_000_000))
    return torch, h


def row_wedges(h, s):
    """W_{s,i} from vertex degrees restricted to E_s (no overlaps involved)."""
    m = h.m
    sizes = np.diff(h.off).astype(np.int64)
    row = np.repeat(np.arange(m, dtype=np.int64), sizes)
    keep = sizes[row] >= s
    v, r = h.idx[keep].astype(np.int64), row[keep]
    order = np.lexsort((r, v))
    vs, rs = v[order], r[order]
    ends = np.searchsorted(vs, vs, side="right")
    later = ends - 1 - np.arange(vs.size)  # entries after this one in adj_s(v)
    w = np.zeros(m, np.int64)
    np.add.at(w, rs, later)
    return w


@pytest.mark.parametrize("s", [1, 4, 8])
def test_medium_full_size_sampled_rows(medium, s):
    torch, h = medium
    dev = torch.device("cuda")
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        pairs, wedges = slg.slg_count(g, s)
        rowoff = slg.slg_row_offsets(g, s)
        counts = np.diff(rowoff)
        assert int(counts.sum()) == pairs
        I = torch.empty(WINDOW, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        digests = torch.zeros(h.m, dtype=torch.int64, device=dev)
        osum = 0
        splits = slg.slg_plan_windows(g, s, WINDOW)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            P, _ = slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, WINDOW,
                                        row_digests=digests[int(r0):int(r1)])
            assert P == rowoff[r1] - rowoff[r0]
            if s == 1:
                osum += int(O[:P].sum(dtype=torch.int64).item())
        dig = digests.cpu().numpy().view(np.uint64)
    finally:
        g.free()

    # rows to check: 1000 seeded random rows + the 100 rows with the most wedges
    rng = np.random.default_rng([7, s])
    sample = rng.choice(h.m, size=1000, replace=False)
    w = row_wedges(h, s)
    heavy = np.argsort(-w, kind="stable")[:100]
    rows = np.unique(np.concatenate([sample, heavy])).astype(np.int32)
    ocount, odig, osum_rows = oracle.rows(h.off, h.idx, rows, [s])
    assert np.array_equal(counts[rows], ocount[:, 0])
    assert np.array_equal(dig[rows], odig[:, 0])
    assert np.array_equal(osum_rows[:, 0], w[rows])  # oracle overlap sums = wedge counts

    deg_s = np.bincount(h.idx[np.repeat(np.diff(h.off) >= s, np.diff(h.off))],
                        minlength=h.n).astype(np.int64)
    assert wedges == int((deg_s * (deg_s - 1) // 2).sum())
    if s == 1:
        # every wedge is one unit of some pair's overlap
        assert osum == wedges


def test_medium_full_size_ensemble(medium):
    """s = 1..8 as one ensemble (Algorithm 3) on the medium workload, one list at
    a time through 2^33-pair windows as the ensemble benchmark runs it: per-row
    counts and digests of every list on 600 seeded random rows and the 50 rows
    with the most wedges equal the oracle's, and each list's row counts add up
    to its |L_s| from the single-s path."""
    torch, h = medium
    dev = torch.device("cuda")
    s_list = list(range(1, 9))
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        pairs, w1 = slg.slg_ensemble_count(g, s_list)
        rowoff = slg.slg_ensemble_row_offsets(g, s_list)
        I = torch.empty(WINDOW, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        digs = []
        for t in range(len(s_list)):
            assert int(rowoff[t, -1]) == pairs[t]
            d = torch.zeros(h.m, dtype=torch.int64, device=dev)
            splits = slg.slg_ensemble_plan_windows(g, s_list, WINDOW, which=t)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                (P,), _ = slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O,
                                                        WINDOW, row_digests=d[int(r0):int(r1)],
                                                        which=t)
                assert P == rowoff[t, r1] - rowoff[t, r0]
            digs.append(d.cpu().numpy().view(np.uint64))
        single = [slg.slg_count(g, s)[0] for s in (1, 5, 8)]
    finally:
        g.free()
    assert single == [pairs[0], pairs[4], pairs[7]]
    rng = np.random.default_rng([7, 99])
    w = row_wedges(h, 1)
    heavy = np.argsort(-w, kind="stable")[:50]
    rows = np.unique(np.concatenate([rng.choice(h.m, size=600, replace=False), heavy]))
    rows = rows.astype(np.int32)
    ocount, odig, osum = oracle.rows(h.off, h.idx, rows, s_list)
    assert np.array_equal(osum[:, 0], w[rows])
    for t in range(len(s_list)):
        assert np.array_equal(np.diff(rowoff[t])[rows], ocount[:, t]), f"list {t}"
        assert np.array_equal(digs[t][rows], odig[:, t]), f"list {t}"


@pytest.fixture(scope="module")
def large():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    h = synth.cached("large_m20000000_seed0", lambda: synth.large(seed=0))
    return torch, h


def test_large_full_size_sampled_rows(large):
    """The large workload (m = 20,000,000, about 2.7e8 incidences), s in
    {2, 4, 8, 16}, through windows of 2^33 pairs: per-row counts and digests of
    120 seeded random rows and the 20 rows with the most wedges at s = 2 equal
    the oracle's; per-row counts add up to |L_s|; W_s matches its closed form."""
    torch, h = large
    dev = torch.device("cuda")
    s_list = [2, 4, 8, 16]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    counts, digs = {}, {}
    try:
        I = torch.empty(WINDOW, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        for s in s_list:
            pairs, wedges = slg.slg_count(g, s)
            rowoff = slg.slg_row_offsets(g, s)
            c = np.diff(rowoff)
            assert int(c.sum()) == pairs
            digests = torch.zeros(h.m, dtype=torch.int64, device=dev)
            splits = slg.slg_plan_windows(g, s, WINDOW)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                P, _ = slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, WINDOW,
                                            row_digests=digests[int(r0):int(r1)])
                assert P == rowoff[r1] - rowoff[r0]
            counts[s] = c
            digs[s] = digests.cpu().numpy().view(np.uint64)
            sz = np.diff(h.off)
            deg_s = np.bincount(h.idx[np.repeat(sz >= s, sz)], minlength=h.n).astype(np.int64)
            assert wedges == int((deg_s * (deg_s - 1) // 2).sum())
    finally:
        g.free()
    rng = np.random.default_rng([7, 20])
    # W_{2,i} (every size is >= 2): for each position p of adj(v), the later
    # entries of adj(v) are wedges of the row at p
    offT, idxT = oracle.transpose(h.off, h.idx, h.n)
    vert = np.repeat(np.arange(h.n, dtype=np.int64), np.diff(offT))
    later = offT[1:][vert] - np.arange(idxT.size, dtype=np.int64) - 1
    w = np.bincount(idxT, weights=later, minlength=h.m)
    heavy = np.argsort(-w, kind="stable")[:20]
    rows = np.unique(np.concatenate([rng.choice(h.m, size=120, replace=False), heavy]))
    rows = rows.astype(np.int32)
    ocount, odig, _ = oracle.rows(h.off, h.idx, rows, s_list)
    for k, s in enumerate(s_list):
        assert np.array_equal(counts[s][rows], ocount[:, k]), f"s={s}"
        assert np.array_equal(digs[s][rows], odig[:, k]), f"s={s}"


def test_large_full_size_one_walk_windows(large):
    """The large workload as its benchmark runs it: one-walk windows of every
    list (s in {2, 4, 8, 16}, windows of 2^33 pairs). The windows cover the rows
    once, in order; the pairs per list add up to the ensemble's |L_s|; and for
    80 seeded random rows and the 20 rows with the most wedges, each list's
    pairs of the row (found in the window by binary search on I) have the
    oracle's count and digest."""
    torch, h = large
    dev = torch.device("cuda")
    s_list = [2, 4, 8, 16]
    rng = np.random.default_rng([7, 21])
    offT, idxT = oracle.transpose(h.off, h.idx, h.n)
    vert = np.repeat(np.arange(h.n, dtype=np.int64), np.diff(offT))
    later = offT[1:][vert] - np.arange(idxT.size, dtype=np.int64) - 1
    w = np.bincount(idxT, weights=later, minlength=h.m)
    heavy = np.argsort(-w, kind="stable")[:20]
    rows = np.unique(np.concatenate([rng.choice(h.m, size=80, replace=False), heavy]))
    rows = rows.astype(np.int32)
    ocount, odig, _ = oracle.rows(h.off, h.idx, rows, s_list)
    got_count = np.zeros((rows.size, len(s_list)), np.int64)
    got_dig = np.zeros((rows.size, len(s_list)), np.uint64)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        I = torch.empty(WINDOW, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        tot = [0] * len(s_list)
        r0, nwin = 0, 0
        while r0 < h.m:
            r1, pairs = slg.slg_ensemble_stream_window(g, s_list, r0, I, J, O, WINDOW)
            assert r0 < r1 <= h.m
            assert sum(pairs) <= WINDOW
            sel = np.flatnonzero((rows >= r0) & (rows < r1))
            b = 0
            for t, p in enumerate(pairs):
                if sel.size and p:
                    seg = I[b:b + p]
                    key = torch.from_numpy(rows[sel]).to(dev)
                    lo = torch.searchsorted(seg, key, right=False).cpu().numpy()
                    hi = torch.searchsorted(seg, key, right=True).cpu().numpy()
                    for x, a, z in zip(sel, lo, hi):
                        got_count[x, t] = z - a
                        got_dig[x, t] = oracle.list_digest(I[b + a:b + z].cpu().numpy(),
                                                           J[b + a:b + z].cpu().numpy(),
                                                           O[b + a:b + z].cpu().numpy())
                tot[t] += p
                b += p
            r0 = r1
            nwin += 1
        assert r0 == h.m and nwin > 1
        want, _ = slg.slg_ensemble_count(g, s_list)
        assert tot == want
    finally:
        g.free()
    for k, s in enumerate(s_list):
        assert np.array_equal(got_count[:, k], ocount[:, k]), f"s={s}"
        assert np.array_equal(got_dig[:, k], odig[:, k]), f"s={s}"


# ------------------------------------------------------- the batched workload

@pytest.fixture(scope="module")
def batch_full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    return torch, [synth.batch_member(b) for b in range(4096)]


def test_batch_full_size_sampled_rows(batch_full):
    """The 4,096-graph batch exactly as the batch benchmark runs it (one batch
    handle, autotuned bins, windows of 2^33 pairs): each member's pair count
    equals its own slg_count, the batch's W is the sum of the members', and
    per-row counts and digests of 1,000 seeded random rows and the 100 rows with
    the most wedges (spread over the members) equal the oracle's on the owning
    member (rows are independent units of Algorithm 2, so sampled rows are a
    sound check)."""
    torch, members = batch_full
    dev = torch.device("cuda")
    hs = [h for h, _ in members]
    s_list = [s for _, s in members]
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    b = slg.slg_batch_load(gs, s_list)
    try:
        slg.slg_autotune(b, 0, max_trials=24)
        pairs, wedges = slg.slg_count(b, 0)
        rb = slg.slg_batch_info(b)
        pb = slg.slg_batch_pair_offsets(b)
        rowoff = slg.slg_row_offsets(b, 0)
        counts = np.diff(rowoff)
        assert int(counts.sum()) == pairs == int(pb[-1])
        I = torch.empty(WINDOW, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        digests = torch.zeros(b.m, dtype=torch.int64, device=dev)
        splits = slg.slg_plan_windows(b, 0, WINDOW)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            P, _ = slg.slg_build_window(b, 0, int(r0), int(r1), I, J, O, WINDOW,
                                        row_digests=digests[int(r0):int(r1)])
            assert P == rowoff[r1] - rowoff[r0]
        dig = digests.cpu().numpy().view(np.uint64)
        del I, J, O
        own_w = 0
        for k, (g, s) in enumerate(zip(gs, s_list)):
            p, w = slg.slg_count(g, s)
            assert int(pb[k + 1] - pb[k]) == p, k
            own_w += w
        assert wedges == own_w
    finally:
        b.free()
        for g in gs:
            g.free()
    # 1000 random rows of the whole batch, and the 100 heaviest rows of the 64
    # largest members (the members of the largest m hold the heaviest rows)
    rng = np.random.default_rng([7, 4096])
    rows = set(rng.choice(int(rb[-1]), size=1000, replace=False).tolist())
    big = np.argsort([-h.m for h in hs], kind="stable")[:64]
    heavy = []
    for k in big:
        w = row_wedges(hs[k], s_list[k])
        top = np.argsort(-w, kind="stable")[:100]
        heavy += [(int(w[i]), int(rb[k]) + int(i)) for i in top]
    rows |= {r for _, r in sorted(heavy, reverse=True)[:100]}
    rows = np.array(sorted(rows), np.int64)
    owner = np.searchsorted(rb, rows, side="right") - 1
    for k in np.unique(owner):
        sel = rows[owner == k]
        h = hs[k]
        oc, od, _ = oracle.rows(h.off, h.idx, (sel - rb[k]).astype(np.int32), [s_list[k]])
        assert np.array_equal(counts[sel], oc[:, 0]), k
        assert np.array_equal(dig[sel], od[:, 0]), k


# -------------------------------------------------------- the served workload

SERVE_CFG = dict(memory_budget=64 << 30, window_pairs=1 << 28, max_result_pairs=1 << 26,
                 workers=8, max_s=16, digest=True, policy=1, small_workers=2,
                 small_wedges=2_000_000_000, batch_max=8)
ORACLE_FULL_M = 40000  # graphs up to this size are checked on every row


def test_served_set_full_size():
    """The 64 resident graphs of the served workload (8 with m = 1,000,000 and 56
    with m log-uniform in [1e3, 1e5]) behind the served benchmark's server
    configuration, with one or two queries per graph submitted together so
    that they mix (and small ones batch). Every query's |L_s| and list digest
    must be exact: against the oracle over all rows for the graphs with m <=
    40,000, and for the larger ones against the library's own windowed build,
    whose per-row counts and digests are then checked against the oracle on
    300 seeded random rows and the 20 rows with the most wedges."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    dev = torch.device("cuda")
    hs = [synth.served_member(g) for g in range(64)]
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    rng = np.random.default_rng([5, 64])
    queries = []
    for g in range(64):
        for s in rng.choice(np.arange(1, 17), size=1 if g < 8 else 2, replace=False):
            queries.append((g, int(s)))
    order = rng.permutation(len(queries))
    got = {}
    try:
        srv = slg.Server(**SERVE_CFG)
        try:
            ids = [slg.slg_serve_register(srv, g) for g in gs]
            tickets = [(queries[q], slg.slg_serve_submit(srv, ids[queries[q][0]], queries[q][1]))
                       for q in order]
            for (g, s), t in tickets:
                r = slg.slg_serve_poll(srv, t, 1_800_000)
                assert r["status"] == 0, (g, s)
                got[(g, s)] = (r["pairs"], r["digest"], r["wedges"])
                slg.slg_serve_release(srv, t)
            st = slg.slg_serve_stats(srv)
        finally:
            srv.close()
        assert st["completed"] == len(queries) and st["batch_failures"] == 0
        # W_s of every query from its closed form
        for (g, s), (_, _, w) in got.items():
            h = hs[g]
            sz = np.diff(h.off)
            deg = np.bincount(h.idx[np.repeat(sz >= s, sz)], minlength=h.n).astype(np.int64)
            assert w == int((deg * (deg - 1) // 2).sum()), (g, s)
        # whole lists against the oracle
        for g in range(64):
            h = hs[g]
            mine = sorted(s for (gg, s) in got if gg == g)
            if h.m > ORACLE_FULL_M:
                continue
            oc, od, _ = oracle.rows(h.off, h.idx, None, mine)
            for t, s in enumerate(mine):
                assert got[(g, s)][0] == int(oc[:, t].sum()), (g, s)
                assert got[(g, s)][1] == int(od[:, t].astype(np.uint64).sum(dtype=np.uint64)), (g, s)
        # the larger graphs: the served result against the windowed build, and the
        # windowed build's sampled rows against the oracle
        win = 1 << 31
        I = torch.empty(win, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        for (g, s) in sorted(got):
            h = hs[g]
            if h.m <= ORACLE_FULL_M:
                continue
            rowoff = slg.slg_row_offsets(gs[g], s)
            digests = torch.zeros(h.m, dtype=torch.int64, device=dev)
            splits = slg.slg_plan_windows(gs[g], s, win)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                slg.slg_build_window(gs[g], s, int(r0), int(r1), I, J, O, win,
                                     row_digests=digests[int(r0):int(r1)])
            dig = digests.cpu().numpy().view(np.uint64)
            counts = np.diff(rowoff)
            assert got[(g, s)][0] == int(counts.sum()), (g, s)
            assert got[(g, s)][1] == int(dig.sum(dtype=np.uint64)), (g, s)
            r2 = np.random.default_rng([7, g, s])
            w = row_wedges(h, s)
            rows = np.unique(np.concatenate([r2.choice(h.m, size=300, replace=False),
                                             np.argsort(-w, kind="stable")[:20]])).astype(np.int32)
            oc, od, _ = oracle.rows(h.off, h.idx, rows, [s])
            assert np.array_equal(counts[rows], oc[:, 0]), (g, s)
            assert np.array_equal(dig[rows], od[:, 0]), (g, s)
    finally:
        for g in gs:
            g.free()
