"""Row-range sharding across two CPU ranks (gloo): slices concatenate to the list.

Each rank computes its row range of L_s(H) (here with the CPU oracle, since the
ranks run without a GPU), the ranks exchange their pair counts, and the slices
placed at the exchanged offsets must form exactly the canonical list.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2201_11326_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, s, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = synth.medium(seed=31, m=2500)
    _, _, osum = oracle.rows(h.off, h.idx, None, [s], nthreads=2)
    splits = shard.balanced_splits(osum[:, 0], world)
    r0, r1 = int(splits[rank]), int(splits[rank + 1])
    rows = np.arange(r0, r1, dtype=np.int32)
    parts = [oracle.row_list(h.off, h.idx, int(i), s) for i in rows]
    I = np.concatenate([np.full(j.size, i, np.int32) for i, (j, _) in zip(rows, parts)] or
                       [np.zeros(0, np.int32)])
    J = np.concatenate([j for j, _ in parts] or [np.zeros(0, np.int32)])
    O = np.concatenate([o for _, o in parts] or [np.zeros(0, np.int32)])
    counts = shard.exchange_counts(I.size)
    base = shard.global_offsets(counts)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), I=I, J=J, O=O, base=base[rank],
             counts=counts, splits=splits)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("s", [1, 3])
def test_two_rank_shards_concatenate(tmp_path, s):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), s, str(tmp_path)), nprocs=world, join=True)
    h = synth.medium(seed=31, m=2500)
    wI, wJ, wO = oracle.slg(h.off, h.idx, s)
    I = np.zeros(wI.size, np.int32)
    J = np.zeros_like(I)
    O = np.zeros_like(I)
    seen = 0
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        b = int(d["base"])
        n = d["I"].size
        assert int(d["counts"][r]) == n
        I[b:b + n], J[b:b + n], O[b:b + n] = d["I"], d["J"], d["O"]
        seen += n
    assert seen == wI.size
    assert np.array_equal(I, wI) and np.array_equal(J, wJ) and np.array_equal(O, wO)


def test_balanced_splits_rules():
    w = np.array([5, 0, 0, 5, 10, 0, 0, 0], np.int64)
    sp = shard.balanced_splits(w, 2)
    assert sp[0] == 0 and sp[-1] == w.size and np.all(np.diff(sp) >= 0)
    assert w[sp[0]:sp[1]].sum() <= 10 and w[sp[1]:].sum() >= 10
    assert shard.balanced_splits(np.zeros(5), 3).tolist() == [0, 1, 3, 5]
    assert shard.global_offsets([3, 0, 4]).tolist() == [0, 3, 3, 7]
