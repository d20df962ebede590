"""Ensembles (Algorithm 3, Section III-D): several s-line graphs of one hypergraph.

Every list of an ensemble must equal the oracle's L_s for its s, element by
element, whatever handler the rows go to; windows and digests must agree with
the single-s path; bad threshold lists are rejected.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg
from tests.test_gpu_parity import FORCED, assert_same
from tests.test_oracle_pins import csr_from_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    torch.cuda.init()


_ORACLE = {}


def oracle_list(key, h, s):
    if (key, s) not in _ORACLE:
        _ORACLE[(key, s)] = oracle.slg_par(h.off, h.idx, s)
    return _ORACLE[(key, s)]


def check_ensemble(h, key, s_list, bins=None):
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        if bins is not None:
            slg.slg_set_bins(g, *bins)
        lists = slg.slg_ensemble_build(g, s_list)
        pairs, wedges = slg.slg_ensemble_count(g, s_list)
    finally:
        g.free()
    assert len(lists) == len(s_list)
    for s, got, p in zip(s_list, lists, pairs):
        want = oracle_list(key, h, s)
        assert p == want[0].size
        assert_same(got, want, f"{key} ensemble {list(s_list)} s={s} bins={bins}")
    return wedges


@pytest.mark.parametrize("mode", sorted(FORCED))
def test_ensemble_medium_recipe_forced_handlers(mode):
    h = synth.medium(seed=2, m=6000)
    check_ensemble(h, "med6000", [1, 2, 3, 5, 8, 13], FORCED[mode])


@pytest.mark.parametrize("mode", ["default", "block_only", "dense_only", "dense_cta_only", "sparse_only"])
def test_ensemble_multitile(mode):
    # hub rows whose partners span several j tiles with a ragged tail
    h = synth.striped_hub(3, 70001, 3000, 40)
    check_ensemble(h, "striped", [1, 2, 3], FORCED[mode])


def test_ensemble_tiny_all_sixteen():
    h = synth.tiny()
    s_list = list(range(1, 17))
    w = check_ensemble(h, "tiny", s_list)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        assert w == slg.slg_count(g, 1)[1]  # W of the smallest threshold
    finally:
        g.free()


@pytest.mark.parametrize("seed", range(4))
def test_ensemble_random_lists(seed):
    rng = np.random.default_rng([11, seed])
    h = synth.uniform_random(seed, 3000, 800, 1, 40)
    k = int(rng.integers(1, 7))
    s_list = sorted(rng.choice(np.arange(1, 12), size=k, replace=False).tolist())
    check_ensemble(h, f"rand{seed}", s_list)


def test_single_threshold_equals_slg_build():
    h = synth.medium(seed=4, m=4000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        for s in (1, 4):
            (got,) = slg.slg_ensemble_build(g, [s])
            assert_same(got, slg.slg_build(g, s), f"s={s}")
    finally:
        g.free()


def test_ensemble_windows_digests_and_row_offsets():
    h = synth.medium(seed=2, m=6000)
    s_list = [2, 3, 6]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        pairs, _ = slg.slg_ensemble_count(g, s_list)
        rowoff = slg.slg_ensemble_row_offsets(g, s_list)
        cap = max(1000, sum(pairs) // 7)
        splits = slg.slg_ensemble_plan_windows(g, s_list, cap)
        assert splits[0] == 0 and splits[-1] == h.m and len(splits) > 2
        parts = [[] for _ in s_list]
        rows_dig = np.zeros((len(s_list), h.m), np.uint64)
        I = np.zeros(cap, np.int32)
        J = np.zeros(cap, np.int32)
        O = np.zeros(cap, np.int32)
        tot_dig = [0] * len(s_list)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            r0, r1 = int(r0), int(r1)
            rd = np.zeros(len(s_list) * (r1 - r0), np.uint64)
            got, dig = slg.slg_ensemble_build_window(g, s_list, r0, r1, I, J, O, cap,
                                                     digest=True, row_digests=rd)
            assert sum(got) <= cap
            b = 0
            for t, p in enumerate(got):
                assert p == rowoff[t, r1] - rowoff[t, r0]
                parts[t].append((I[b:b + p].copy(), J[b:b + p].copy(), O[b:b + p].copy()))
                b += p
                tot_dig[t] = (tot_dig[t] + dig[t]) % (1 << 64)
            rows_dig[:, r0:r1] = rd.reshape(len(s_list), r1 - r0)
        for t, s in enumerate(s_list):
            want = oracle_list("med6000", h, s)
            got = tuple(np.concatenate([p[c] for p in parts[t]]) for c in range(3))
            assert_same(got, want, f"windows s={s}")
            assert np.array_equal(np.diff(rowoff[t]), np.bincount(want[0], minlength=h.m))
            assert tot_dig[t] == oracle.list_digest(*want)
            # the single-s path gives the same row digests
            single = np.zeros(h.m, np.uint64)
            Is = np.zeros(max(pairs[t], 1), np.int32)
            Js, Os = np.zeros_like(Is), np.zeros_like(Is)
            slg.slg_build_window(g, s, 0, h.m, Is, Js, Os, row_digests=single)
            assert np.array_equal(single, rows_dig[t])
    finally:
        g.free()


@pytest.mark.parametrize("mode", ["default", "dense_only", "dense_cta_only", "block_only", "sparse_only"])
def test_ensemble_one_list_at_a_time(mode):
    # which = t: list t alone, in its own windows, from the shared plan
    h = synth.medium(seed=2, m=6000)
    s_list = [1, 2, 4, 7]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        slg.slg_set_bins(g, *FORCED[mode])
        pairs, _ = slg.slg_ensemble_count(g, s_list)
        for t, s in enumerate(s_list):
            cap = max(500, pairs[t] // 5)
            splits = slg.slg_ensemble_plan_windows(g, s_list, cap, which=t)
            I = np.zeros(cap, np.int32)
            J = np.zeros(cap, np.int32)
            O = np.zeros(cap, np.int32)
            parts, tot = [], 0
            for r0, r1 in zip(splits[:-1], splits[1:]):
                (p,), (d,) = slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O,
                                                           cap, digest=True, which=t)
                parts.append((I[:p].copy(), J[:p].copy(), O[:p].copy()))
                tot = (tot + d) % (1 << 64)
            want = oracle_list("med6000", h, s)
            got = tuple(np.concatenate([x[c] for x in parts]) for c in range(3))
            assert_same(got, want, f"list {t} s={s} {mode}")
            assert tot == oracle.list_digest(*want)
        with pytest.raises(slg.SlgError) as e:
            slg.slg_ensemble_plan_windows(g, s_list, 100, which=len(s_list))
        assert e.value.code == slg.SLG_EINVAL
    finally:
        g.free()


def test_ensemble_device_buffers():
    import torch
    h = synth.medium(seed=3, m=5000)
    s_list = [1, 4]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        pairs, _ = slg.slg_ensemble_count(g, s_list)
        tot = sum(pairs)
        dev = torch.device("cuda")
        I = torch.empty(tot, dtype=torch.int32, device=dev)
        J = torch.empty_like(I)
        O = torch.empty_like(I)
        rd = torch.zeros(len(s_list) * h.m, dtype=torch.int64, device=dev)
        got, _ = slg.slg_ensemble_build_window(g, s_list, 0, h.m, I, J, O, tot, row_digests=rd)
        assert got == pairs
        b = 0
        for s, p in zip(s_list, pairs):
            want = oracle.slg(h.off, h.idx, s)
            assert_same((I[b:b + p].cpu().numpy(), J[b:b + p].cpu().numpy(),
                         O[b:b + p].cpu().numpy()), want, f"device s={s}")
            b += p
    finally:
        g.free()


def test_ensemble_and_single_calls_interleave():
    # the cached plan must follow whichever call came last
    h = synth.medium(seed=5, m=3000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        a = slg.slg_ensemble_build(g, [1, 3])
        one = slg.slg_build(g, 1)
        three = slg.slg_build(g, 3)
        b = slg.slg_ensemble_build(g, [1, 3])
        c = slg.slg_ensemble_build(g, [3, 5])
        five = slg.slg_build(g, 5)
    finally:
        g.free()
    for x, y in ((a[0], one), (a[1], three), (b[0], one), (b[1], three), (c[0], three),
                 (c[1], five)):
        assert_same(x, y)
    assert_same(one, oracle.slg(h.off, h.idx, 1))
    assert_same(c[1], oracle.slg(h.off, h.idx, 5))


def test_ensemble_edge_cases():
    # empty graphs and rows, duplicates, one hub row, thresholds above every overlap
    cases = {
        "empty_graph": ([], 5),
        "all_empty_rows": ([[], [], []], 4),
        "one_row": ([[0, 1, 2]], 3),
        "duplicates": ([[1, 2, 3]] * 5 + [[2, 3]] * 3, 4),
        "hub_row": ([list(range(300))] + [[v] for v in range(300)] + [list(range(0, 300, 2))],
                    300),
        "singletons": ([[v % 7] for v in range(50)], 7),
    }
    s_list = [1, 2, 3, 200]
    for name, (rows, n) in cases.items():
        off, idx = csr_from_rows(rows)
        h = synth.Hypergraph(off, idx, n)
        g = slg.slg_load(h.off, h.idx, h.m, h.n)
        try:
            lists = slg.slg_ensemble_build(g, s_list)
        finally:
            g.free()
        for s, got in zip(s_list, lists):
            assert_same(got, oracle.slg(off, idx, s), f"{name} s={s}")


def test_ensemble_rejects_bad_lists():
    h = synth.tiny()
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        for bad in ([], [2, 2], [3, 1], [0, 1], list(range(1, 18)), [-1]):
            with pytest.raises(slg.SlgError) as e:
                slg.slg_ensemble_count(g, bad)
            assert e.value.code == slg.SLG_EINVAL
        # too small a buffer: SLG_ECAPACITY, pairs still reported
        pairs, _ = slg.slg_ensemble_count(g, [1, 2])
        I = np.zeros(1, np.int32)
        with pytest.raises(slg.SlgError) as e:
            slg.slg_ensemble_build_window(g, [1, 2], 0, h.m, I, I.copy(), I.copy(), 1)
        assert e.value.code == slg.SLG_ECAPACITY
    finally:
        g.free()
    g1 = slg.slg_load(h.off, h.idx, h.m, h.n)
    b = slg.slg_batch_load([g1], [1])
    try:
        with pytest.raises(slg.SlgError) as e:
            slg.slg_ensemble_count(b, [1, 2])
        assert e.value.code == slg.SLG_EINVAL
    finally:
        b.free()
        g1.free()


@pytest.mark.parametrize("handler", ["hubpair", "sparse"])
def test_ensemble_one_walk_large_recipe(handler):
    # up to four lists: the sparse-accumulator and hub-pair rows are walked once
    # for every list (one counting launch each), the other handlers per list
    h = synth.large(m=20000)
    s_list = [2, 3, 5, 8]
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    mode = slg.MODE_NAMES.index(handler)
    try:
        if handler == "hubpair":
            slg.slg_set_bins(g, *FORCED["block_only"])
            slg.slg_set_hub_pairs(g, 512, 0)
        else:
            slg.slg_set_bins(g, *FORCED["sparse_cta_only"])
            slg.slg_set_hub_pairs(g, 0, 0)
        slg.slg_set_timing(g, True)
        slg.slg_kernel_stats(g, reset=True)
        pairs, _ = slg.slg_ensemble_count(g, s_list)
        assert slg.slg_kernel_stats(g)[1][0][mode] == 1
        assert slg.slg_ensemble_mode_stats(g, s_list, 0)[mode][0] > 0
        counts, digs, _ = oracle.rows(h.off, h.idx, None, s_list)
        assert pairs == [int(x) for x in counts.sum(axis=0)]
        for s, got in zip(s_list, slg.slg_ensemble_build(g, s_list)):
            assert_same(got, oracle_list("large20000", h, s), f"{handler} s={s}")
        for t in range(len(s_list)):
            cap = max(int(counts[:, t].max()), int(counts[:, t].sum()) // 3 + 1)
            I, J, O = (np.zeros(cap, np.int32) for _ in range(3))
            splits = slg.slg_ensemble_plan_windows(g, s_list, cap, which=t)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                rd = np.zeros(r1 - r0, np.uint64)
                slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap=cap,
                                              digest=True, row_digests=rd, which=t)
                assert np.array_equal(rd, digs[r0:r1, t]), (handler, t, r0)
        # five lists go back to one launch per list
        slg.slg_kernel_stats(g, reset=True)
        slg.slg_ensemble_count(g, [2, 3, 5, 8, 13])
        assert slg.slg_kernel_stats(g)[1][0][mode] == 5
    finally:
        g.free()


@pytest.mark.parametrize("mode", [-1, 0, 1])
def test_ensemble_lists_filtered_from_the_one_before(mode):
    # windows of every list: a later list walked, or filtered from the list before
    # it (the lists are nested and in the same order); the same lists either way
    h = synth.large(m=20000)
    s_list = [2, 3, 5, 8]
    counts, digs, _ = oracle.rows(h.off, h.idx, None, s_list)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        slg.slg_set_hub_pairs(g, 512, 0)
        slg.slg_set_ensemble_filter(g, mode)
        for s, got in zip(s_list, slg.slg_ensemble_build(g, s_list)):
            assert_same(got, oracle_list("large20000", h, s), f"filter {mode} s={s}")
        tot = counts.sum(axis=1)
        cap = max(int(tot.max()), int(tot.sum()) // 4 + 1)
        I, J, O = (np.zeros(cap, np.int32) for _ in range(3))
        splits = slg.slg_ensemble_plan_windows(g, s_list, cap)
        assert len(splits) > 2
        slg.slg_ensemble_fill_stats(g, reset=True)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            nr = int(r1 - r0)
            rd = np.zeros(len(s_list) * nr, np.uint64)
            got, _ = slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap,
                                                   digest=True, row_digests=rd)
            assert got == [int(x) for x in counts[r0:r1].sum(axis=0)]
            for t in range(len(s_list)):
                assert np.array_equal(rd[t * nr:(t + 1) * nr], digs[r0:r1, t]), (mode, t, r0)
        # how each list was made: every window either walked or filtered it, the
        # first list always walked, and the pairs add up to the list's
        made = slg.slg_ensemble_fill_stats(g)
        nwin = len(splits) - 1
        for t in range(len(s_list)):
            assert made[t][0] + made[t][2] == nwin, (mode, t, made[t])
            assert made[t][1] + made[t][3] == int(counts[:, t].sum()), (mode, t, made[t])
        assert made[0][2] == 0
        if mode == 0:
            assert not made[1:, 2].any()
        if mode == 1:
            assert not made[1:len(s_list), 0].any()
            for t in range(1, len(s_list)):  # each filter read the whole list before
                assert made[t][5] == int(counts[:, t - 1].sum()), (t, made[t])
        assert not made[:, 4].any()         # filter times only while timing is on
        assert not made[len(s_list):].any()
        with pytest.raises(slg.SlgError):
            slg.slg_set_ensemble_filter(g, 2)
    finally:
        g.free()
