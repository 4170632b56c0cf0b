"""ubqp_solve_rounds: R independent rounds of one instance run together (one
evaluation launch over all R*S starts, one climb launch over every round's
passing starts).  Round k must equal ubqp_solve with seed + k and
loop-counter offset round + k, and the oracle's round with the same starts."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def oracle_round(Q, S, lam, seed, round_, mode):
    """One round of Fig. 2's loop body from the oracle's pinned pieces."""
    n = Q.shape[0]
    X = orc.diversify(orc.first_derivative(Q), n, mode, seed, round_, S)
    f = orc.eval(Q, X)
    sc = orc.screen(f, lam)
    Xa, fa, _ = orc.ascent(Q, X, f, sc["idx"])
    bf, bi = orc.best(fa)
    return bf, bi, Xa[bi]


@pytest.mark.parametrize("n,density,S,R,mode", [
    (100, 0.1, 1000, 3, ubqp.DIVERSIFY),
    (257, 0.5, 300, 5, ubqp.RANDOM),
    (1500, 1.0, 500, 4, ubqp.DIVERSIFY),
    (2500, 0.1, 1000, 1, ubqp.RANDOM),
    (7000, 1.0, 1000, 3, ubqp.RANDOM),     # the n = 7000 workload, three rounds in flight
])
def test_rounds_equal_separate_solves(n, density, S, R, mode):
    Q = synth.make_instance(n, density, 60 + n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    lam, seed = 0.5, 9
    p = ubqp.make_params(S, lam, mode=mode, seed=seed)
    bx, bf = ubqp.solve_rounds(inst, p, R)
    inst.sync()
    for k in range(R):
        pk = ubqp.make_params(S, lam, mode=mode, seed=seed + k, round_=k)
        sx, sf, _ = ubqp.solve(inst, pk, want_stats=False)
        inst.sync()
        assert torch.equal(bf[k], sf) and torch.equal(bx[k], sx), k
        if n <= 1500:
            wf, wi, wx = oracle_round(Q, S, lam, seed + k, k, mode)
            assert [int(bf[k, 0]), int(bf[k, 1])] == [wf, wi], k
            assert np.array_equal(bx[k].cpu().numpy().view(np.uint64), wx), k


def test_rounds_argument_errors():
    Q = synth.make_instance(64, 0.5, 1)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    p = ubqp.make_params(100, 0.5)
    assert ubqp.solve_rounds_workspace_size(inst, p, 0) == 0
    assert ubqp.solve_rounds_workspace_size(inst, p, 1025) == 0
    with pytest.raises(ubqp.UbqpError):
        ubqp.solve_rounds(inst, p, 2, ws=torch.empty(16, dtype=torch.uint8, device="cuda"))
