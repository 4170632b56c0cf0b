"""The multi-round search of Fig. 2 on the device against the oracle's."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,density,S,rounds,lam", [(100, 0.1, 64, 6, 0.5),
                                                     (300, 0.5, 100, 4, 0.25),
                                                     (1000, 1.0, 40, 3, 0.75)])
def test_search_matches_oracle(n, density, S, rounds, lam):
    Q = synth.make_instance(n, density, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    got = ubqp.search(inst, num_samples=500, starts_per_round=S, rounds=rounds, lam=lam,
                      seed=7)
    inst.sync()
    want = orc.search(Q, 500, S, rounds, lam, seed=7)
    assert int(got["best_f"].item()) == want["best_f"]
    assert np.array_equal(got["best_x"].cpu().numpy().view(np.uint64), want["best_x"])
    assert got["history"].cpu().tolist() == want["history"].tolist()
    assert got["stats"].cpu().tolist() == [want["passed"], want["total_flips"], want["sample_sum"]]


def test_search_zero_rounds_returns_first_derivative_start():
    n = 200
    Q = synth.make_instance(n, 0.3, 1)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    got = ubqp.search(inst, num_samples=10, starts_per_round=8, rounds=0, lam=0.5)
    x0 = orc.first_derivative(Q)
    assert np.array_equal(got["best_x"].cpu().numpy().view(np.uint64), x0)
    assert int(got["best_f"].item()) == orc.f(Q, x0)


@pytest.mark.parametrize("split", [0, 3, 7])
def test_search_resume_equals_one_search(split):
    """Checkpoint/resume: rounds 0..R-1 in one call equal rounds 0..split-1
    followed by a resumption from the saved state for the rest."""
    n, S, R = 300, 256, 7
    Q = synth.make_instance(n, 0.5, 12)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    kw = dict(num_samples=500, starts_per_round=S, lam=0.4, seed=21)
    whole = ubqp.search(inst, rounds=R, **kw)
    first = ubqp.search(inst, rounds=split, **kw)
    rest = ubqp.search_resume(inst, first, split, rounds=R - split, **kw)
    inst.sync()
    assert torch.equal(rest["best_x"], whole["best_x"])
    assert torch.equal(rest["best_f"], whole["best_f"])
    assert torch.equal(rest["stats"], whole["stats"])
    hist = torch.cat([first["history"], rest["history"]])
    assert torch.equal(hist, whole["history"])


@pytest.mark.parametrize("lam", [float("nan"), float("inf")])
def test_search_rejects_non_finite_lambda(lam):
    """T(lambda) needs a finite lambda: the call fails before any round."""
    Q = synth.make_instance(64, 0.5, 2)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    with pytest.raises(ubqp.UbqpError) as e:
        ubqp.search(inst, num_samples=10, starts_per_round=8, rounds=2, lam=lam)
    assert e.value.status == -1  # UBQP_ERR_ARG
