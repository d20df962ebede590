"""The served form: concurrent queries over resident graphs, admission, results.

Every query's result (kept list or streamed digest) must equal the oracle's,
whether it runs alone or mixed with other queries on other workers.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graphs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    hs = [synth.tiny(), synth.medium(seed=21, m=4000), synth.striped_hub(8, 6000, 500, 30),
          synth.served_member(9), synth.uniform_random(4, 300, 100, 1, 10)]
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    yield hs, gs
    for g in gs:
        g.free()


def oracle_digest(h, s):
    _, dig, _ = oracle.rows(h.off, h.idx, None, [s])
    return int(dig[:, 0].astype(np.uint64).sum(dtype=np.uint64))


def test_mixed_queries_match_oracle(graphs):
    hs, gs = graphs
    srv = slg.Server(memory_budget=8 << 30, window_pairs=1 << 22, max_result_pairs=1 << 22,
                     workers=4, max_s=8, policy=1, small_workers=1, small_wedges=10_000_000)
    try:
        ids = [slg.slg_serve_register(srv, g) for g in gs]
        rng = np.random.default_rng(3)
        queries = [(int(rng.integers(0, len(gs))), int(rng.integers(1, 9))) for _ in range(40)]
        tickets = [slg.slg_serve_submit(srv, ids[g], s) for g, s in queries]
        for t, (g, s) in zip(tickets, queries):
            r = slg.slg_serve_poll(srv, t, 120000)
            h = hs[g]
            wI, wJ, wO = oracle.slg_par(h.off, h.idx, s)
            assert r["pairs"] == wI.size and r["status"] == 0
            assert r["digest"] == oracle.list_digest(wI, wJ, wO)
            if r["materialized"]:
                I, J, O = slg.slg_serve_fetch(srv, t, r["pairs"])
                assert np.array_equal(I, wI) and np.array_equal(J, wJ) and np.array_equal(O, wO)
            slg.slg_serve_release(srv, t)
        st = slg.slg_serve_stats(srv)
        assert st["completed"] == len(queries) and st["p99_us"] >= st["p50_us"] > 0
        assert st["peak_memory"] <= 8 << 30
    finally:
        srv.close()


def test_same_result_alone_and_in_the_mix(graphs):
    hs, gs = graphs
    target = (1, 2)
    alone = slg.Server(4 << 30, 1 << 20, 1 << 26, workers=1, max_s=8)
    mixed = slg.Server(4 << 30, 1 << 20, 1 << 26, workers=6, max_s=8)
    try:
        a_ids = [slg.slg_serve_register(alone, g) for g in gs]
        m_ids = [slg.slg_serve_register(mixed, g) for g in gs]
        ta = slg.slg_serve_submit(alone, a_ids[target[0]], target[1])
        ra = slg.slg_serve_poll(alone, ta, 120000)
        assert ra["materialized"] == 1
        la = slg.slg_serve_fetch(alone, ta, ra["pairs"])
        others = [slg.slg_serve_submit(mixed, m_ids[g], s) for g in range(len(gs)) for s in (1, 3)]
        tm = slg.slg_serve_submit(mixed, m_ids[target[0]], target[1])
        others += [slg.slg_serve_submit(mixed, m_ids[g], 2) for g in range(len(gs))]
        rm = slg.slg_serve_poll(mixed, tm, 120000)
        lm = slg.slg_serve_fetch(mixed, tm, rm["pairs"])
        assert ra["digest"] == rm["digest"] and ra["pairs"] == rm["pairs"]
        assert all(np.array_equal(x, y) for x, y in zip(la, lm))
        for t in others:
            assert slg.slg_serve_poll(mixed, t, 120000)["status"] == 0
    finally:
        alone.close()
        mixed.close()


def test_streamed_results_and_admission(graphs):
    hs, gs = graphs
    # results above 1000 pairs are streamed through 5000-pair windows
    srv = slg.Server(memory_budget=200_000, window_pairs=5000, max_result_pairs=1000, workers=3,
                     max_s=4)
    try:
        ids = [slg.slg_serve_register(srv, g) for g in gs]
        t = slg.slg_serve_submit(srv, ids[0], 1)
        r = slg.slg_serve_poll(srv, t, 120000)
        assert r["materialized"] == 0
        assert r["digest"] == oracle_digest(hs[0], 1)
        # a kept result larger than the budget could never be admitted
        small = slg.Server(memory_budget=100, window_pairs=5000, max_result_pairs=1 << 20,
                           workers=1, max_s=4)
        try:
            gid = slg.slg_serve_register(small, gs[0])
            with pytest.raises(slg.SlgError) as ei:
                slg.slg_serve_submit(small, gid, 3)  # kept (< 2^20 pairs), > 100 bytes
            assert ei.value.code == slg.SLG_ECAPACITY
        finally:
            small.close()
    finally:
        srv.close()


def test_large_query_reaches_a_general_worker(graphs):
    # with workers restricted to small queries, a large query must still run
    hs, gs = graphs
    srv = slg.Server(1 << 30, 1 << 20, 1 << 24, workers=3, max_s=4, policy=1, small_workers=2,
                     small_wedges=1)
    try:
        gid = slg.slg_serve_register(srv, gs[1])
        for _ in range(3):
            t = slg.slg_serve_submit(srv, gid, 2)
            assert slg.slg_serve_poll(srv, t, 60000)["status"] == 0
            slg.slg_serve_release(srv, t)
    finally:
        srv.close()


def test_poll_timeout(graphs):
    hs, gs = graphs
    srv = slg.Server(1 << 30, 1 << 20, 1 << 24, workers=1, max_s=4)
    try:
        gid = slg.slg_serve_register(srv, gs[1])
        first = slg.slg_serve_submit(srv, gid, 1)
        second = slg.slg_serve_submit(srv, gid, 2)
        with pytest.raises(slg.SlgError) as ei:
            slg.slg_serve_poll(srv, second, 0)
        assert ei.value.code == slg.SLG_ETIMEOUT
        assert slg.slg_serve_poll(srv, first, 120000)["status"] == 0
        assert slg.slg_serve_poll(srv, second, 120000)["status"] == 0
    finally:
        srv.close()


def test_batched_small_queries_match_oracle(graphs):
    # continuous batching: small queries of different graphs and s run as one batch;
    # each result (kept list, pairs, W_s, digest) must be what it is alone
    hs, gs = graphs
    srv = slg.Server(memory_budget=8 << 30, window_pairs=1 << 24, max_result_pairs=1 << 22,
                     workers=2, max_s=8, policy=1, small_workers=1, small_wedges=1 << 40,
                     batch_max=8)
    try:
        ids = [slg.slg_serve_register(srv, g) for g in gs]
        rng = np.random.default_rng(17)
        queries = [(int(rng.integers(0, len(gs))), int(rng.integers(1, 9))) for _ in range(48)]
        tickets = [slg.slg_serve_submit(srv, ids[g], s) for g, s in queries]
        sizes = []
        for t, (g, s) in zip(tickets, queries):
            r = slg.slg_serve_poll(srv, t, 120000)
            sizes.append(r["batch_size"])
            h = hs[g]
            wI, wJ, wO = oracle.slg_par(h.off, h.idx, s)
            assert r["status"] == 0 and r["pairs"] == wI.size, (g, s)
            assert r["digest"] == oracle.list_digest(wI, wJ, wO), (g, s)
            sz = np.diff(h.off)
            deg = np.bincount(h.idx[np.repeat(sz >= s, sz)], minlength=h.n).astype(np.int64)
            assert r["wedges"] == int((deg * (deg - 1) // 2).sum()), (g, s)
            if r["materialized"]:
                I, J, O = slg.slg_serve_fetch(srv, t, r["pairs"])
                assert np.array_equal(I, wI) and np.array_equal(J, wJ) and np.array_equal(O, wO)
            slg.slg_serve_release(srv, t)
        st = slg.slg_serve_stats(srv)
        assert st["completed"] == len(queries)
        # batches really formed, and none failed over to one-by-one runs
        assert st["batch_failures"] == 0, st.get("batch_error")
        assert st["batches"] > 0 and st["batched"] == sum(1 for x in sizes if x > 1)
        assert max(sizes) > 1
    finally:
        srv.close()
