"""The seeded generators: determinism, CSR shape rules, and the recipe's marginals."""
import numpy as np

import oracle
import synth


def test_deterministic_and_valid():
    a = synth.tiny()
    b = synth.tiny()
    assert np.array_equal(a.off, b.off) and np.array_equal(a.idx, b.idx)
    assert a.m == 2000 and a.n == 1000
    assert oracle.validate(a.off, a.idx, a.n)
    sz = a.sizes()
    assert sz.min() >= 2 and sz.max() <= 100


def test_medium_recipe_scaled():
    h = synth.medium(m=20000)
    assert h.n == 10000 and oracle.validate(h.off, h.idx, h.n)
    sz = h.sizes()
    assert sz.min() >= 2 and sz.max() <= 5000
    # log-normal(1.8, 1.0): median of exp(N) is e^1.8 ~ 6
    assert 5 <= np.median(sz) <= 7
    # Zipf(1.7) popularity: the top vertex has ~49% of the draw mass, so it sits
    # in most hyperedges
    deg = np.bincount(h.idx, minlength=h.n)
    assert deg.max() > 0.6 * h.m


def test_chunks_are_independent():
    # rows of chunk 0 do not depend on how many rows follow
    a = synth.build((3,), 1000, 500, "lognormal", (1.8, 1.0, 2, 50), "zipf", (1.7,))
    b = synth.build((3,), 1000, 500, "lognormal", (1.8, 1.0, 2, 50), "zipf", (1.7,))
    assert np.array_equal(a.idx, b.idx)


def test_batch_and_served_members():
    g, s = synth.batch_member(5)
    assert 100 <= g.m <= 100000 and 1 <= s <= 4 and g.n == g.m // 2
    assert oracle.validate(g.off, g.idx, g.n)
    h = synth.served_member(9)
    assert 1000 <= h.m <= 100000


def test_save_load_roundtrip(tmp_path):
    h = synth.tiny()
    p = str(tmp_path / "t.csr")
    synth.save(h, p)
    g = synth.load(p)
    assert np.array_equal(h.off, g.off) and np.array_equal(h.idx, g.idx) and g.n == h.n


def test_fast_member_draw():
    # the C draw follows the same rule: valid rows of the requested sizes,
    # deterministic per seed, Zipf(1.7) hubs in most rows
    a = synth.build((4,), 20000, 10000, "lognormal", (1.8, 1.0, 2, 5000), "zipf", (1.7,),
                    fast=True)
    b = synth.build((4,), 20000, 10000, "lognormal", (1.8, 1.0, 2, 5000), "zipf", (1.7,),
                    fast=True)
    assert np.array_equal(a.idx, b.idx) and oracle.validate(a.off, a.idx, a.n)
    ref = synth.build((4,), 20000, 10000, "lognormal", (1.8, 1.0, 2, 5000), "zipf", (1.7,))
    assert np.array_equal(a.sizes(), ref.sizes())  # same size stream
    da, dr = np.bincount(a.idx, minlength=a.n), np.bincount(ref.idx, minlength=ref.n)
    assert abs(int(da.max()) - int(dr.max())) < 0.02 * a.m
    assert set(np.argsort(-da)[:3].tolist()) == set(np.argsort(-dr)[:3].tolist())
