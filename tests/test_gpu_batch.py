"""Batches of uneven instances: every instance's result equals its single
solve (and the oracle's), with the default, the autotuned and the captured-
graph execution."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def make_batch(sizes, densities, seed0=100):
    Qs, insts = [], []
    for k, (n, d) in enumerate(zip(sizes, densities)):
        Q = synth.make_instance(n, d, seed0 + k)
        Qs.append(Q)
        insts.append(ubqp.Instance(torch.from_numpy(Q).cuda()))
    return Qs, insts


def check_against_single(insts, batch, params, seed):
    for i, inst in enumerate(insts):
        bx, bf = batch.result(i)
        p1 = ubqp.make_params(params.num_starts, params.lambda_, mode=params.mode, seed=seed,
                              eval_path=params.eval_path)
        sx, sf, _ = ubqp.solve(inst, p1, want_stats=False)
        torch.cuda.synchronize()
        assert torch.equal(bf, sf), (i, bf.tolist(), sf.tolist())
        assert torch.equal(bx, sx), i


SIZES = [60, 700, 2500, 300, 1025, 129, 2100, 513]
DENS = [1.0, 0.1, 0.5, 1.0, 0.1, 0.5, 1.0, 0.1]


@pytest.mark.parametrize("mode", [ubqp.DIVERSIFY, ubqp.RANDOM])
def test_batch_equals_single_solves(mode):
    Qs, insts = make_batch(SIZES, DENS)
    p = ubqp.make_params(256, 0.5, mode=mode, seed=1)
    b = ubqp.Batch(insts, p)
    b.run(seed=5)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 5)
    # the small instances against the oracle too
    for i in (0, 5):
        want = orc.solve(Qs[i], 256, 0.5, seed=5, mode=mode)
        bx, bf = b.result(i)
        assert int(bf[0]) == want["best_f"] and int(bf[1]) == want["best_index"]
        assert np.array_equal(bx.cpu().numpy().view(np.uint64), want["best_x"])


def test_batch_tune_and_graph_keep_results():
    Qs, insts = make_batch(SIZES, DENS, seed0=300)
    p = ubqp.make_params(300, 0.25, seed=2)
    b = ubqp.Batch(insts, p)
    b.tune()
    cfg = b.config()
    assert cfg["asc_threads"] * cfg["asc_chunks"] * 16 >= max(SIZES)
    b.run(seed=7)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 7)
    b.capture()
    assert b.config()["graph"] == 1
    for seed in (11, 12):  # replays with new seeds
        b.run(seed=seed)
        torch.cuda.synchronize()
        check_against_single(insts, b, p, seed)


def test_batch_plain_eval_path():
    Qs, insts = make_batch([200, 900, 1500], [0.5, 1.0, 0.1], seed0=500)
    p = ubqp.make_params(128, 0.5, seed=3, eval_path=ubqp.EVAL_PLAIN)
    b = ubqp.Batch(insts, p)
    assert b.config()["eval_path"] == ubqp.EVAL_PLAIN
    b.run(seed=9)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 9)


@pytest.mark.parametrize("shape,packed,kch,merged", [
    ((256, 1), True, 16, True), ((256, 2), True, 8, True), ((256, 1), False, 12, False),
    ((128, 2), False, 8, True), ((256, 1), True, 12, False)])
def test_batch_pinned_schedules_equal_single_solves(shape, packed, kch, merged):
    # packed climbs (sub-groups of 32 / 64 / 128 / 256 threads by n, several starts
    # of one instance per block) and every evaluation schedule give the same
    # results as single solves, with the graph too
    sizes = [60, 700, 2500, 300, 1025, 129, 2100, 513, 1024, 1023, 2048, 2049]
    dens = [1.0, 0.1, 0.5, 1.0, 0.1, 0.5, 1.0, 0.1, 0.5, 1.0, 0.1, 0.5]
    Qs, insts = make_batch(sizes, dens, seed0=700)
    p = ubqp.make_params(257, 0.3, seed=4)
    b = ubqp.Batch(insts, p)
    b.set(shape[0], shape[1], packed=packed, eval_kch=kch, eval_merged=merged)
    cfg = b.config()
    assert (cfg["asc_threads"], cfg["asc_chunks"], cfg["packed"], cfg["eval_kch"],
            cfg["eval_merged"]) == (shape[0], shape[1], int(packed), kch, int(merged))
    b.run(seed=21)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 21)
    b.capture()
    b.run(seed=22)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 22)
    for i in (0, 3):
        want = orc.solve(Qs[i], 257, 0.3, seed=22)
        bx, bf = b.result(i)
        assert int(bf[0]) == want["best_f"] and int(bf[1]) == want["best_index"]
        assert np.array_equal(bx.cpu().numpy().view(np.uint64), want["best_x"])


def test_batch_set_rejects_shapes_that_cannot_hold_n():
    Qs, insts = make_batch([3000, 100], [0.5, 0.5], seed0=900)
    b = ubqp.Batch(insts, ubqp.make_params(64, 0.5, seed=1))
    with pytest.raises(ubqp.UbqpError):
        b.set(128, 1)          # 2048 elements < 3000
    with pytest.raises(ubqp.UbqpError):
        b.set(128, 2, packed=True)  # packed blocks are 256 threads
    with pytest.raises(ubqp.UbqpError):
        b.set(256, 1, eval_kch=5)
    bp = ubqp.Batch(insts, ubqp.make_params(64, 0.5, seed=1, eval_path=ubqp.EVAL_PLAIN))
    with pytest.raises(ubqp.UbqpError):
        bp.set(256, 1, eval_merged=True)  # the merged launch is the tensor-core path


def test_batch_merged_evaluation_values():
    # one merged launch each for the start generation and the evaluation of
    # instances of ragged sizes (single words, word and tile tails, and sizes
    # where single solves take the staged evaluation), at every schedule:
    # results equal to single solves
    sizes = [60, 700, 2500, 300, 1025, 129, 2100, 513, 1, 64, 65, 4096, 4100]
    Qs, insts = make_batch(sizes, [0.5] * len(sizes), seed0=950)
    p = ubqp.make_params(300, 0.5, seed=0)
    b = ubqp.Batch(insts, p)
    b.set(256, 2, packed=True, eval_kch=16, eval_merged=True)
    b.run(seed=31)
    torch.cuda.synchronize()
    check_against_single(insts, b, p, 31)
    for kch in (12, 8):
        b.set(256, 2, packed=True, eval_kch=kch, eval_merged=True)
        b.run(seed=32)
        torch.cuda.synchronize()
        check_against_single(insts, b, p, 32)
