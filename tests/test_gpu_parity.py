"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, bit-exact.

Every case compares the full canonical list (I, J, O) element by element, or,
at full size, per-row counts and digests of sampled rows plus totals fixed by
closed forms.
"""
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg
from tests.test_oracle_pins import csr_from_rows, parse_golden

pytestmark = pytest.mark.gpu

# bin settings that force one handler onto every row (results must not change)
FORCED = {
    # (warp_max_wedges, block_item_wedges, dense_min_density, dense_item_tiles,
    #  wdense_max_ranges, sparse_min_per_tile, sparse_item_wedges, wsparse_max_size)
    "default": (128, 1024, 64, 4, 32, 64, 65536, 32),
    "block_only": (0, 1024, -1, 4, 32, -1, 65536, 32),
    "block_one_item_per_row": (0, 1 << 30, -1, 4, 32, -1, 65536, 32),  # big items: split path
    "block_tiny_items": (0, 1, -1, 4, 32, -1, 65536, 32),
    "dense_only": (0, 1024, 0, 1, 32, -1, 65536, 32),           # warp-level dense where possible
    "dense_cta_only": (0, 1024, 0, 1, 0, -1, 65536, 32),        # CTA-level dense for every dense row
    "dense_warp_few_ranges": (0, 1024, 0, 3, 2, -1, 65536, 32),  # warp dense only for <= 2 ranges
    "warp_and_block": (128, 256, -1, 4, 32, -1, 65536, 32),
    "sparse_only": (0, 1024, -1, 4, 32, 0, 65536, 32),          # warp sparse (|e| <= 32), else CTA
    "sparse_cta_only": (0, 1024, -1, 4, 32, 0, 65536, 0),       # CTA sparse for |e| <= 255
    "sparse_tiny_items": (0, 1024, -1, 4, 32, 0, 1, 32),        # one item per 1024 ids
    "sparse_and_dense": (128, 1024, 64, 4, 32, 0, 4096, 32),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    torch.cuda.init()


def gpu_list(h, s, bins=None):
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        if bins is not None:
            slg.slg_set_bins(g, *bins)
        return slg.slg_build(g, s)
    finally:
        g.free()


def assert_same(got, want, ctx=""):
    gI, gJ, gO = got
    wI, wJ, wO = want
    assert gI.size == wI.size, f"{ctx}: {gI.size} pairs vs oracle {wI.size}"
    for name, a, b in (("I", gI, wI), ("J", gJ, wJ), ("O", gO, wO)):
        if not np.array_equal(a, b):
            k = int(np.flatnonzero(a != b)[0])
            raise AssertionError(f"{ctx}: {name} differs first at {k}: "
                                 f"gpu ({gI[k]},{gJ[k]},{gO[k]}) oracle ({wI[k]},{wJ[k]},{wO[k]})")


def test_worked_example(golden_dir):
    n, rows, pairs, *_ = parse_golden(os.path.join(golden_dir, "worked_example.txt"))
    off, idx = csr_from_rows(rows)
    h = synth.Hypergraph(off, idx, n)
    for s in range(1, 6):
        I, J, O = gpu_list(h, s)
        assert list(zip(I.tolist(), J.tolist(), O.tolist())) == sorted(pairs.get(s, []))


def test_transpose_matches_oracle():
    for h in (synth.tiny(), synth.medium(m=20000), synth.uniform_random(1, 500, 300, 0, 9)):
        g = slg.slg_load(h.off, h.idx, h.m, h.n)
        offT, idxT = slg.slg_transpose_copy(g)
        g.free()
        wo, wi = oracle.transpose(h.off, h.idx, h.n)
        assert np.array_equal(offT, wo) and np.array_equal(idxT, wi)


@pytest.mark.parametrize("s", [1, 2, 3])
def test_tiny_workload(s):
    h = synth.tiny()
    assert_same(gpu_list(h, s), oracle.slg(h.off, h.idx, s), f"tiny s={s}")


@pytest.mark.parametrize("mode", sorted(FORCED))
def test_forced_handlers_tiny(mode):
    h = synth.tiny()
    for s in (1, 2, 3):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle.slg(h.off, h.idx, s), f"{mode} s={s}")


_ORACLE_CACHE = {}


def oracle_list(key, h, s):
    if (key, s) not in _ORACLE_CACHE:
        _ORACLE_CACHE[(key, s)] = oracle.slg_par(h.off, h.idx, s)
    return _ORACLE_CACHE[(key, s)]


@pytest.mark.parametrize("mode", sorted(FORCED))
def test_forced_handlers_medium_recipe(mode):
    # the medium workload's recipe (Zipf hubs in most rows), scaled down
    h = synth.medium(seed=2, m=6000)
    for s in (1, 3, 8):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle_list("med6000", h, s), f"{mode} s={s}")


@pytest.mark.parametrize("mode", sorted(FORCED))
def test_forced_handlers_multitile(mode):
    # hub rows whose partners span three 32768-wide j tiles and a ragged tail
    h = synth.striped_hub(3, 70001, 3000, 40)
    for s in (1, 2):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle_list("striped", h, s), f"{mode} s={s}")


def _overflow_graph():
    # row 0 holds vertices 0 and 1: its partners are every 5th and every 7th
    # row of one 65536-id tile, more than the 8192 touched counters a sparse
    # tile lists, so that tile's survivors are read off the whole tile
    m = 65000
    rng = np.random.default_rng(9)
    rows = []
    for i in range(m):
        r = set(int(x) for x in rng.choice(np.arange(2, 400), size=int(rng.integers(1, 4)),
                                           replace=False))
        if i % 5 == 0:
            r.add(0)
        if i % 7 == 0:
            r.add(1)
        rows.append(sorted(r))
    off, idx = csr_from_rows(rows)
    return synth.Hypergraph(off, idx, 400)


@pytest.mark.parametrize("mode", ["sparse_only", "sparse_cta_only", "sparse_tiny_items", "default"])
def test_sparse_touched_list_overflow(mode):
    h = _overflow_graph()
    for s in (1, 2):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle_list("overflow", h, s), f"{mode} s={s}")


@pytest.mark.parametrize("mode", ["default", "sparse_only", "sparse_cta_only", "sparse_and_dense",
                                  "block_only"])
def test_large_recipe_scaled_down(mode):
    # the large workload's recipe (Chung-Lu, degrees Zipf(1.8) capped at 1e5,
    # log-normal sizes up to 20000) at m = 20000, s as in that workload
    h = synth.large(m=20000)
    for s in (2, 4, 8, 16):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle_list("large20000", h, s), f"{mode} s={s}")


@pytest.mark.parametrize("seed", range(6))
def test_random_small(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 400))
    n = int(rng.integers(1, 300))
    h = synth.uniform_random(seed, m, n, 0, min(n, 40))
    for s in (1, 2, 4, 7):
        assert_same(gpu_list(h, s), oracle.slg(h.off, h.idx, s), f"seed={seed} s={s}")


def test_count_and_wedges():
    h = synth.medium(seed=4, m=30000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    sizes = h.sizes()
    row = np.repeat(np.arange(h.m), sizes)
    s_list = list(range(1, 9))
    counts, _, _ = oracle.rows(h.off, h.idx, None, s_list)
    for t, s in enumerate(s_list):
        pairs, wedges = slg.slg_count(g, s)
        ds = np.bincount(h.idx[sizes[row] >= s], minlength=h.n).astype(np.int64)
        assert wedges == int((ds * (ds - 1) // 2).sum())
        assert pairs == int(counts[:, t].sum())
        assert slg.slg_bound(g, s) >= pairs
        rowoff = slg.slg_row_offsets(g, s)
        assert np.array_equal(np.diff(rowoff), counts[:, t])
    g.free()


def test_edge_cases():
    cases = {
        "empty_graph": ([], 5),
        "all_empty_rows": ([[], [], []], 4),
        "one_row": ([[0, 1, 2]], 3),
        "duplicates": ([[1, 2, 3]] * 5 + [[2, 3]] * 3, 4),
        "hub_row": ([list(range(300))] + [[v] for v in range(300)] + [list(range(0, 300, 2))], 300),
        "singletons": ([[v % 7] for v in range(50)], 7),
    }
    for name, (rows, n) in cases.items():
        off, idx = csr_from_rows(rows)
        h = synth.Hypergraph(off, idx, n)
        for s in (1, 2, 3, 200):
            assert_same(gpu_list(h, s), oracle.slg(off, idx, s), f"{name} s={s}")


def test_hub_masks_many_hubs():
    # more than 32 high-degree vertices, rows holding every hub, hub-only rows
    rng = np.random.default_rng(21)
    n = 400
    rows = []
    for i in range(3000):
        k = int(rng.integers(1, 12))
        r = set(rng.choice(60, size=min(k, 60), replace=False).tolist())  # 60 popular vertices
        r |= set(rng.choice(np.arange(60, n), size=int(rng.integers(0, 4)), replace=False).tolist())
        rows.append(sorted(r))
    rows += [list(range(64))] * 3 + [list(range(0, 64, 2))]
    off, idx = csr_from_rows(rows)
    h = synth.Hypergraph(off, idx, n)
    for s in (1, 2, 5, 9):
        want = oracle.slg(off, idx, s)
        for mode in ("default", "dense_only", "dense_cta_only", "block_only"):
            assert_same(gpu_list(h, s, FORCED[mode]), want, f"{mode} s={s}")


def test_s_clique_graphs_through_the_dual():
    for h in (synth.tiny(), synth.medium(seed=15, m=3000)):
        g = slg.slg_load(h.off, h.idx, h.m, h.n)
        d = slg.slg_dual(g)
        try:
            assert (d.m, d.n, d.nnz) == (h.n, h.m, h.nnz)
            offT, idxT = oracle.transpose(h.off, h.idx, h.n)
            for s in (1, 2, 4):
                assert_same(slg.slg_build(d, s), oracle.slg_par(offT, idxT, s), f"dual s={s}")
        finally:
            d.free()
            g.free()


def test_invalid_input_rejected():
    bad = {
        "unsorted": (np.array([0, 2], np.int32), np.array([3, 1], np.int32), 1, 4),
        "repeat": (np.array([0, 2], np.int32), np.array([1, 1], np.int32), 1, 4),
        "range": (np.array([0, 1], np.int32), np.array([4], np.int32), 1, 4),
        "negative": (np.array([0, 1], np.int32), np.array([-1], np.int32), 1, 4),
        "offsets": (np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), 2, 4),
        "off0": (np.array([1, 2], np.int32), np.array([0, 1], np.int32), 1, 4),
    }
    for name, (off, idx, m, n) in bad.items():
        with pytest.raises(slg.SlgError) as ei:
            slg.slg_load(off, idx, m, n)
        assert ei.value.code == slg.SLG_EINVAL, name
    h = synth.tiny()
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    with pytest.raises(slg.SlgError) as ei:
        slg.slg_count(g, 0)
    assert ei.value.code == slg.SLG_EINVAL
    I = np.zeros(3, np.int32)
    with pytest.raises(slg.SlgError) as ei:
        slg.slg_build(g, 1, I, I.copy(), I.copy(), cap=3)
    assert ei.value.code == slg.SLG_ECAPACITY
    g.free()


def test_windows_and_digests():
    h = synth.medium(seed=6, m=5000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    for s in (1, 4):
        wI, wJ, wO = oracle.slg_par(h.off, h.idx, s)
        counts, digs, _ = oracle.rows(h.off, h.idx, None, [s])
        cap = max(int(counts.max()), wI.size // 7 + 1)
        splits = slg.slg_plan_windows(g, s, cap)
        assert splits[0] == 0 and splits[-1] == h.m and np.all(np.diff(splits) > 0)
        I = np.zeros(cap, np.int32)
        J = np.zeros(cap, np.int32)
        O = np.zeros(cap, np.int32)
        parts, total = [], 0
        for r0, r1 in zip(splits[:-1], splits[1:]):
            rd = np.zeros(r1 - r0, np.uint64)
            P, d = slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, digest=True,
                                        row_digests=rd)
            assert P <= cap
            parts.append((I[:P].copy(), J[:P].copy(), O[:P].copy()))
            total = (total + d) % 2**64
            assert np.array_equal(rd, digs[r0:r1, 0])
        got = tuple(np.concatenate([p[k] for p in parts]) for k in range(3))
        assert_same(got, (wI, wJ, wO), f"windows s={s}")
        assert total == oracle.list_digest(wI, wJ, wO)
    g.free()


def test_device_buffers_and_stream():
    import torch
    h = synth.medium(seed=7, m=5000)
    st = torch.cuda.Stream()
    off = torch.from_numpy(h.off).cuda()
    idx = torch.from_numpy(h.idx).cuda()
    g = slg.slg_load(off, idx, h.m, h.n, stream=st)
    pairs, _ = slg.slg_count(g, 2)
    I = torch.empty(pairs, dtype=torch.int32, device="cuda")
    J = torch.empty_like(I)
    O = torch.empty_like(I)
    slg.slg_build(g, 2, I, J, O)
    st.synchronize()
    want = oracle.slg_par(h.off, h.idx, 2)
    assert_same((I.cpu().numpy(), J.cpu().numpy(), O.cpu().numpy()), want, "device buffers")
    g.free()


def test_repeated_calls_are_identical():
    h = synth.medium(seed=8, m=8000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    a = slg.slg_build(g, 2)
    slg.slg_count(g, 5)
    b = slg.slg_build(g, 2)
    assert_same(a, b, "rebuild")
    g.free()


# ------------------------------------------------------------------ batches


def _batch_members():
    hs = [synth.tiny(seed=3), synth.medium(seed=12, m=3000), synth.striped_hub(5, 9000, 700, 50),
          synth.uniform_random(9, 200, 150, 0, 12)]
    for b in range(12):
        g, s = synth.batch_member(b)
        if g.m <= 6000:
            hs.append(g)
    rng = np.random.default_rng(5)
    s_list = [int(x) for x in rng.integers(1, 5, size=len(hs))]
    return hs, s_list


@pytest.mark.parametrize("mode", ["default", "block_only", "dense_only", "dense_cta_only", "sparse_only"])
def test_batch_members_equal_their_own_lists(mode):
    hs, s_list = _batch_members()
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    b = slg.slg_batch_load(gs, s_list)
    try:
        slg.slg_set_bins(b, *FORCED[mode])
        rb = slg.slg_batch_info(b)
        assert rb.tolist() == np.concatenate([[0], np.cumsum([h.m for h in hs])]).tolist()
        pairs, wedges = slg.slg_count(b, 0)
        pb = slg.slg_batch_pair_offsets(b)
        I, J, O = slg.slg_build(b, 0)
        assert pb[-1] == pairs == I.size
        tot_w = 0
        for k, (h, s) in enumerate(zip(hs, s_list)):
            want = oracle.slg(h.off, h.idx, s)
            sl = slice(int(pb[k]), int(pb[k + 1]))
            assert_same((I[sl], J[sl], O[sl]), want, f"member {k} s={s}")
            tot_w += slg.slg_count(gs[k], s)[1]
        assert wedges == tot_w
        # digests of the batch equal the members' own
        rd = np.zeros(b.m, np.uint64)
        cap = max(int(pb[-1]), 1)
        Iw, Jw, Ow = (np.zeros(cap, np.int32) for _ in range(3))
        slg.slg_build_window(b, 0, 0, b.m, Iw, Jw, Ow, cap, row_digests=rd)
        for k, h in enumerate(hs):
            _, dig, _ = oracle.rows(h.off, h.idx, None, [s_list[k]])
            assert np.array_equal(rd[rb[k]:rb[k + 1]], dig[:, 0]), k
        with pytest.raises(slg.SlgError):
            slg.slg_count(b, 2)
    finally:
        b.free()
        for g in gs:
            g.free()


def test_autotune_keeps_results():
    # the autotuner only changes how rows are binned; lists must stay identical
    h = synth.medium(seed=2, m=6000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        bins, ms = slg.slg_autotune(g, 2, max_trials=8)
        assert len(bins) == 8 and ms > 0
        assert bins[3] >= 1 and bins[6] >= 1
        assert_same(slg.slg_build(g, 2), oracle_list("med6000", h, 2), f"autotuned {bins}")
        assert_same(slg.slg_build(g, 3), oracle_list("med6000", h, 3), f"autotuned {bins}")
        with pytest.raises(slg.SlgError) as e:
            slg.slg_autotune(g, 0, max_trials=4)
        assert e.value.code == slg.SLG_EINVAL
    finally:
        g.free()


def test_autotune_batch_handle():
    hs, s_list = _batch_members()
    graphs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    b = slg.slg_batch_load(graphs, s_list)
    try:
        bins, _ = slg.slg_autotune(b, 0, max_trials=6)
        base = slg.slg_batch_pair_offsets(b)
        I, J, O = slg.slg_build(b, 0)
        for k, (h, s) in enumerate(zip(hs, s_list)):
            got = (I[base[k]:base[k + 1]], J[base[k]:base[k + 1]], O[base[k]:base[k + 1]])
            assert_same(got, oracle.slg(h.off, h.idx, s), f"member {k} autotuned {bins}")
    finally:
        b.free()
        for g in graphs:
            g.free()


def test_output_arrays_at_any_alignment():
    # I, J and O as slices of one buffer at offsets 0, 1 and 3 ints: the fill may
    # not assume that they share an alignment
    import torch
    h = synth.medium(seed=2, m=6000)
    want = oracle_list("med6000", h, 1)
    P = want[0].size
    buf = torch.zeros(3 * P + 8, dtype=torch.int32, device="cuda")
    I, J, O = buf[0:P], buf[P + 1:2 * P + 1], buf[2 * P + 3:3 * P + 3]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        got, _ = slg.slg_build_window(g, 1, 0, h.m, I, J, O, P)
    finally:
        g.free()
    assert got == P
    assert_same((I.cpu().numpy(), J.cpu().numpy(), O.cpu().numpy()), want, "offset slices")


@pytest.mark.parametrize("mode", ["default", "sparse_only", "sparse_cta_only"])
def test_counter_width_boundaries(mode):
    # rows at the 8-bit counters' limit: copies of a 255-vertex row (overlap 255 fits
    # a byte), copies of a 256-vertex row (too large for the sparse accumulators:
    # the binning sends them elsewhere), 32-vertex copies for the warp accumulator,
    # all spread over a wide id range so that they count as sparse rows
    rng = np.random.default_rng(12)
    n = 3000
    big255 = sorted(rng.choice(n, 255, replace=False).tolist())
    big256 = sorted(rng.choice(n, 256, replace=False).tolist())
    mid32 = sorted(rng.choice(n, 32, replace=False).tolist())
    rows = []
    for r in range(20000):
        if r in (5, 10000, 19990):
            rows.append(big255)
        elif r in (7, 15000):
            rows.append(big256)
        elif r in (9, 7500, 19999):
            rows.append(mid32)
        else:
            rows.append(sorted(rng.choice(n, int(rng.integers(1, 4)), replace=False).tolist()))
    off, idx = csr_from_rows(rows)
    h = synth.Hypergraph(off, idx, n)
    for s in (1, 2, 32, 255, 256):
        assert_same(gpu_list(h, s, FORCED[mode]), oracle_list("width", h, s), f"{mode} s={s}")


def test_slg_batch_call_matches_oracle():
    # the one-call batch: per member |L_s|, W_s, digest and (when asked) the list
    hs, s_list = _batch_members()
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    try:
        want = [k % 2 == 0 for k in range(len(hs))]
        res = slg.slg_batch(gs, s_list, want_lists=want)
        assert len(res) == len(hs)
        for k, (h, s, r) in enumerate(zip(hs, s_list, res)):
            wI, wJ, wO = oracle.slg(h.off, h.idx, s)
            assert r["status"] == 0 and r["pairs"] == wI.size, k
            assert r["digest"] == oracle.list_digest(wI, wJ, wO), k
            sz = np.diff(h.off)
            deg = np.bincount(h.idx[np.repeat(sz >= s, sz)], minlength=h.n).astype(np.int64)
            assert r["wedges"] == int((deg * (deg - 1) // 2).sum()), k
            if want[k]:
                assert_same((r["I"], r["J"], r["O"]), (wI, wJ, wO), f"slg_batch member {k}")
            else:
                assert "I" not in r
        # a bad threshold fails the whole call with every status set
        with pytest.raises(slg.SlgError) as ei:
            slg.slg_batch(gs, [0] * len(gs))
        assert ei.value.code == slg.SLG_EINVAL
    finally:
        for g in gs:
            g.free()


def test_slg_batch_windows_smaller_than_the_list():
    # a member list that spans several of the call's device windows (at most 2^27
    # pairs each): two copies of a graph whose s = 1 list has 1.9e8 pairs
    h = synth.medium(seed=3, m=20000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        pairs, _ = slg.slg_count(g, 1)
        assert pairs > (1 << 27)
        res = slg.slg_batch([g, g], [1, 6], want_lists=[True, False])
        counts, digs, _ = oracle.rows(h.off, h.idx, None, [1, 6])
        for k, col in ((0, 0), (1, 1)):
            assert res[k]["pairs"] == int(counts[:, col].sum())
            assert res[k]["digest"] == int(digs[:, col].astype(np.uint64).sum(dtype=np.uint64))
        I, J, O = res[0]["I"], res[0]["J"], res[0]["O"]
        rowoff = np.concatenate([[0], np.cumsum(counts[:, 0])])
        rng = np.random.default_rng(8)
        for i in rng.choice(h.m, size=60, replace=False).tolist() + [0, h.m - 1]:
            wj, wo = oracle.row_list(h.off, h.idx, i, 1)
            a, b = int(rowoff[i]), int(rowoff[i + 1])
            assert np.all(I[a:b] == i) and np.array_equal(J[a:b], wj) and np.array_equal(O[a:b], wo)
    finally:
        g.free()


# ---------------------------------------------------------------- hub pairs

HUBPAIR_GRAPHS = {
    "large20000": lambda: synth.large(m=20000),
    "med6000": lambda: synth.medium(seed=2, m=6000),
    "tiny": lambda: synth.tiny(),
    "striped": lambda: synth.striped_hub(3, 70001, 3000, 40),
    "overflow": _overflow_graph,
}


def hubpair_rows(g, s):
    return slg.slg_mode_stats(g, s)[slg.MODE_NAMES.index("hubpair")][0]


@pytest.mark.parametrize("max_hubs", [2, 16, 256, 4096])
@pytest.mark.parametrize("key", sorted(HUBPAIR_GRAPHS))
def test_hub_pairs_match_oracle(key, max_hubs):
    # partners from non-hub wedges and hub-pair lists (overlap = non-hub count +
    # the hubs recovered from the pair count, or the one-hub check), with and
    # without the table and dense handlers beside them
    h = HUBPAIR_GRAPHS[key]()
    used = 0
    for bins in (None, FORCED["block_only"]):
        g = slg.slg_load(h.off, h.idx, h.m, h.n)
        try:
            if bins is not None:
                slg.slg_set_bins(g, *bins)
            slg.slg_set_hub_pairs(g, max_hubs, 0)
            for s in (2, 3, 5):
                got = slg.slg_build(g, s)
                used += hubpair_rows(g, s)
                assert_same(got, oracle_list(key, h, s), f"{key} hubs<={max_hubs} s={s}")
            # s = 1 never uses hub pairs (a single shared hub is an overlap)
            assert hubpair_rows(g, 1) == 0
        finally:
            g.free()
    if key in ("large20000", "med6000") and max_hubs >= 16:
        assert used > 0


def test_hub_pairs_in_an_ensemble_and_windows():
    h = synth.large(m=20000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        slg.slg_set_bins(g, *FORCED["block_only"])
        slg.slg_set_hub_pairs(g, 512, 0)
        s_list = [2, 4, 8, 16]
        lists = slg.slg_ensemble_build(g, s_list)
        for s, got in zip(s_list, lists):
            assert_same(got, oracle_list("large20000", h, s), f"ensemble s={s}")
        # windows with per-row digests through the hub-pair handler
        counts, digs, _ = oracle.rows(h.off, h.idx, None, [3])
        cap = max(int(counts.max()), int(counts.sum()) // 5 + 1)
        I, J, O = (np.zeros(cap, np.int32) for _ in range(3))
        splits = slg.slg_plan_windows(g, 3, cap)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            rd = np.zeros(r1 - r0, np.uint64)
            slg.slg_build_window(g, 3, int(r0), int(r1), I, J, O, digest=True, row_digests=rd)
            assert np.array_equal(rd, digs[r0:r1, 0])
        assert hubpair_rows(g, 3) > 0
    finally:
        g.free()


def test_hub_pairs_disabled_and_default_threshold():
    h = synth.large(m=20000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        # the default threshold (2^33 sparse wedges) is far above this graph's
        assert hubpair_rows(g, 2) == 0
        slg.slg_set_hub_pairs(g, 0, 0)  # disabled
        assert hubpair_rows(g, 2) == 0
        assert_same(slg.slg_build(g, 2), oracle_list("large20000", h, 2), "disabled")
        with pytest.raises(slg.SlgError):
            slg.slg_set_hub_pairs(g, 5000, 0)
    finally:
        g.free()


# staging pools: automatic, capped (made at any size), none, and one of three
# chunks (spent after three CTAs' worth of items: the counting kernels take the
# others)
@pytest.mark.parametrize("handler", ["hubpair", "sparse"])
@pytest.mark.parametrize("pool", ["auto", "capped", "off", "three_chunks"])
def test_staged_counting_pass(handler, pool):
    # the sparse-accumulator and hub-pair fill kernels run as the counting pass,
    # staging each item's pairs; windows copy staged items and fill the rest
    h = synth.large(m=20000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    mode = slg.MODE_NAMES.index(handler)
    try:
        if handler == "hubpair":
            slg.slg_set_bins(g, *FORCED["block_only"])
            slg.slg_set_hub_pairs(g, 512, 0)
        else:
            slg.slg_set_bins(g, *FORCED["sparse_cta_only"])
            slg.slg_set_hub_pairs(g, 0, 0)
        if pool != "auto":
            slg.slg_set_staging(g, 1 << 34)  # a capped pool is made at any size
            slg.slg_count(g, 2)
            st = slg.slg_staging_stats(g)
            assert st["pool_pairs"] > 0 and st["items_staged"] > 0, st
            # 8 bytes per item, 5 per pooled pair (setting it again releases the
            # counted plan, so the loop below counts again)
            slg.slg_set_staging(g, 1 << 34 if pool == "capped" else 0 if pool == "off" else
                                8 * st["items"] + 5 * 3 * st["chunk_pairs"])
        slg.slg_set_timing(g, True)
        for s in (2, 4, 8):
            slg.slg_kernel_stats(g, reset=True)
            got = slg.slg_build(g, s)
            assert_same(got, oracle_list("large20000", h, s), f"{handler} {pool} s={s}")
            launches = slg.slg_kernel_stats(g)[1][0][mode]
            ms = slg.slg_mode_stats(g, s)
            rows = ms[mode][0]
            st = slg.slg_staging_stats(g)
            assert rows > 0
            staged = st["pool_pairs"] > 0
            if pool == "auto":
                # made only when the rows can fill 2^26 pairs: their wedges (sparse
                # accumulator) and walked entries (hub pairs)
                bound = ms[slg.MODE_NAMES.index("sparse")][1] + \
                    ms[slg.MODE_NAMES.index("hubpair")][4]
                assert staged == (bound >= 1 << 26), (bound, st)
            else:
                assert staged == (pool != "off"), st
            # staging launches the fill kernel before the counting kernel
            assert launches == (2 if staged else 1), (pool, s, launches)
            if pool == "off":
                assert st["items_staged"] == 0
            elif pool == "three_chunks":
                assert 0 < st["items_staged"] and st["pool_pairs"] <= 3 << 20, st
                if s == 2:  # the pool ran out: fewer items staged than the handler's rows
                    assert st["items_staged"] < rows, (st, rows)
        # several windows, each mixing copied and walked items, with row digests
        counts, digs, _ = oracle.rows(h.off, h.idx, None, [3])
        cap = max(int(counts.max()), int(counts.sum()) // 7 + 1)
        I, J, O = (np.zeros(cap, np.int32) for _ in range(3))
        splits = slg.slg_plan_windows(g, 3, cap)
        assert len(splits) > 3
        for r0, r1 in zip(splits[:-1], splits[1:]):
            rd = np.zeros(r1 - r0, np.uint64)
            slg.slg_build_window(g, 3, int(r0), int(r1), I, J, O, digest=True, row_digests=rd)
            assert np.array_equal(rd, digs[r0:r1, 0])
        with pytest.raises(slg.SlgError):
            slg.slg_set_staging(g, -2)
    finally:
        g.free()


