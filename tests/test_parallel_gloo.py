"""The sharded-batch exchanges on two CPU ranks (gloo): partition, the screen
statistics and the best-of must equal the single-rank (oracle) results."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as orc
from paper_1706_00037_gb300 import parallel

WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, S_total, fv, tie_best):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        b, c = parallel.shard(S_total, WORLD, rank)
        loc = fv[b:b + c]
        # per-rank statistics as the stats kernel defines them
        st = torch.tensor([int(loc.sum()), int(loc.max()), b + int(np.argmax(loc))],
                          dtype=torch.int64)
        g = parallel.reduce_screen_stats(st)
        want = orc.screen(fv, 0.5)
        assert [int(v) for v in g] == [want["sum"], want["max"], want["argmax"]], (list(g), want)
        # best-of with the owner's solution words
        bi = int(np.argmax(tie_best[b:b + c]))
        vi = torch.tensor([int(tie_best[b + bi]), b + bi], dtype=torch.int64)
        x = torch.full((3,), 1000 + b + bi, dtype=torch.int64)
        v, idx, xw = parallel.reduce_best(vi, x, S_total)
        wv, wi = orc.best(tie_best)
        assert (v, idx) == (wv, wi)
        assert xw.tolist() == [1000 + wi] * 3
        assert parallel.owner_of(wi, S_total, WORLD) in range(WORLD)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("S_total", [1001, 7])
def test_sharded_exchanges_match_single_rank(S_total):
    r = np.random.default_rng(S_total)
    fv = r.integers(-10**9, 10**9, S_total).astype(np.int64)
    fv[S_total - 1] = fv.max() + 5
    fv[1] = fv[S_total - 1]  # the max on both ranks: the lower index must win
    tie = r.integers(0, 50, S_total).astype(np.int64)
    tie[[0, S_total - 1]] = 99  # a best tied across the ranks
    mp.start_processes(_worker, args=(_free_port(), S_total, fv, tie), nprocs=WORLD,
                       join=True, start_method="spawn")


def test_shard_partition():
    for S in (1, 2, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            got = [parallel.shard(S, world, r) for r in range(world)]
            assert sum(c for _, c in got) == S
            assert got[0][0] == 0
            for (b0, c0), (b1, _) in zip(got, got[1:]):
                assert b1 == b0 + c0
            assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_pure_combinations():
    st = [torch.tensor([10, 7, 3]), torch.tensor([-4, 7, 1]), torch.tensor([5, 2, 9])]
    assert parallel.combine_screen_stats(st).tolist() == [11, 7, 1]
    assert parallel.combine_best([(5, 8), (9, 4), (9, 2)]) == (9, 2)


def test_a_rank_without_starts_is_neutral():
    # more ranks than starts: the empty rank's triple and best change nothing
    empty = torch.tensor([0, parallel.INT64_MIN, parallel.INT64_MAX])
    st = [torch.tensor([-30, -7, 1]), empty, torch.tensor([-5, -2, 2])]
    assert parallel.combine_screen_stats(st).tolist() == [-35, -2, 2]
    assert parallel.combine_best([(-3, 0), (parallel.INT64_MIN, 3), (-3, 1)]) == (-3, 0)
    assert [parallel.shard(2, 3, r) for r in range(3)] == [(0, 1), (1, 1), (2, 0)]
