"""A batch split over two ranks, run on one GPU one rank after the other
(no waiting between kernels), gives exactly the single-rank round."""
import numpy as np
import pytest
import torch

from paper_1706_00037_gb300 import parallel, synth, ubqp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,n,S", [(ubqp.DIVERSIFY, 300, 777), (ubqp.RANDOM, 2100, 500),
                                      (ubqp.RANDOM, 300, 2)])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_round_equals_single_round(mode, n, S, world):
    Q = synth.make_instance(n, 0.3, 5)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    p = ubqp.make_params(S, 0.5, mode=mode, seed=11)
    bx, bf, st = ubqp.solve(inst, p)
    states = [parallel.round_phase1(inst, p, world, r) for r in range(world)]
    g = parallel.combine_screen_stats([s.stats for s in states])
    assert g.tolist() == [st["sum"], st["batch_max"], int(g[2])]
    outs = [parallel.round_phase2(inst, p, s, g) for s in states]
    v, idx = parallel.combine_best([(int(o[0][0]), int(o[0][1])) for o in outs])
    assert (v, idx) == (int(bf[0]), int(bf[1]))
    owner = parallel.owner_of(idx, S, world)
    assert torch.equal(outs[owner][1], bx)
    assert sum(int(o[2]["count"].item()) for o in outs) == st["passed"]
    assert all(float(o[2]["Tm"][0].item()) == st["T"] for o in outs)


def test_diversify_range_is_a_slice():
    n, S = 500, 300
    Q = synth.make_instance(n, 0.3, 5)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    for mode in (ubqp.RANDOM, ubqp.DIVERSIFY):
        full = ubqp.diversify(inst, S, mode=mode, seed=3, round_=2)
        part = ubqp.diversify_range(inst, S, 101, 57, mode=mode, seed=3, round_=2)
        assert torch.equal(full[101:158], part)
