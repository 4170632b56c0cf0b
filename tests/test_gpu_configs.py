"""Parity at the workloads' full sizes, on sampled outputs.

The oracle is too slow to evaluate or climb every start of a full-size batch,
so these tests run the CUDA path exactly as bench.py launches it and check
(a) sampled starts' objective values and ascents against the oracle, run on
inputs the oracle generates itself, and (b) properties that hold at any size
(the screen's pass set against its own threshold, best-of against the batch).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def words_host(t):
    return t.cpu().numpy().view(np.uint64)


def run_round(inst, S, lam, mode, seed, path=ubqp.EVAL_AUTO):
    X = ubqp.diversify(inst, S, mode=mode, seed=seed)
    f = ubqp.eval(inst, X, path=path)
    f0 = f.clone()
    sc = ubqp.screen(f, lam)
    flips = torch.zeros(S, dtype=torch.int32, device="cuda")
    X0 = X.clone()
    ubqp.ascent(inst, X, f, sc["idx"], sc["count"], 0, flips)
    bx, bf = ubqp.best(f, X)
    inst.sync()
    c = int(sc["count"].item())
    return dict(X0=words_host(X0), X=words_host(X), f0=f0.cpu().numpy(), f=f.cpu().numpy(),
                idx=sc["idx"][:c].cpu().numpy(), T=float(sc["Tm"][0].item()),
                mean=float(sc["Tm"][1].item()), stats=sc["stats"].cpu().numpy(),
                flips=flips.cpu().numpy(), bx=words_host(bx), bf=bf.cpu().numpy())


def check_round(Q, n, S, lam, mode, seed, r, x0, n_eval=4, n_climb=2):
    rng = np.random.default_rng(seed)
    Xh = orc.diversify(x0, n, mode, seed, 0, S)
    assert np.array_equal(r["X0"], Xh)  # start generation is cheap: check all
    pick = np.unique(np.concatenate([[0, S - 1], rng.integers(0, S, n_eval)]))
    assert np.array_equal(r["f0"][pick], orc.eval(Q, Xh[pick]))
    # screen: properties at any size
    f0 = r["f0"]
    assert r["stats"][1] == f0.max() and r["stats"][2] == int(np.argmax(f0))
    assert r["stats"][0] == int(f0.sum())
    assert r["mean"] == float(np.float64(int(f0.sum())) / np.float64(S))
    assert list(r["idx"]) == [b for b in range(S) if float(f0[b]) > r["T"]]
    # ascent of sampled passers against the oracle
    if len(r["idx"]):
        for s in rng.choice(r["idx"], size=min(n_climb, len(r["idx"])), replace=False):
            f_s = orc.eval(Q, Xh[s:s + 1])[0]
            xw, fw, cw, _ = orc.ascent1(Q, Xh[s], int(f_s))
            assert int(r["f"][s]) == fw and int(r["flips"][s]) == cw
            assert np.array_equal(r["X"][s], xw)
    # starts that did not pass are untouched
    rest = np.setdiff1d(np.arange(S), r["idx"])
    assert np.array_equal(r["f"][rest], f0[rest]) and np.array_equal(r["X"][rest], Xh[rest])
    # best of the batch
    assert int(r["bf"][0]) == r["f"].max() and int(r["bf"][1]) == int(np.argmax(r["f"]))
    assert np.array_equal(r["bx"], r["X"][int(r["bf"][1])])


def test_table1_dense_n7000_bench_workload():
    # the benchmark's workload: n = 7000, density 1.0, 1000 random starts, lambda 0.5
    n, S, lam = 7000, 1000, 0.5
    Q = synth.make_instance(n, 1.0, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    seed = 1_000_003 + 3
    r = run_round(inst, S, lam, ubqp.RANDOM, seed)
    check_round(Q, n, S, lam, orc.RANDOM, seed, r, None)
    # the plain CUDA-core evaluation agrees on every start
    X = torch.from_numpy(r["X0"].view(np.int64)).cuda()
    assert np.array_equal(ubqp.eval(inst, X, path=ubqp.EVAL_PLAIN).cpu().numpy(), r["f0"])


@pytest.mark.parametrize("lam", [0.25, 0.5, 0.75])
def test_one_large_sparse_instance(lam):
    # n = 5000, density 0.1, 8192 starts diversified around the first-derivative start
    n, S = 5000, 8192
    Q = synth.make_instance(n, 0.1, 3)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    r = run_round(inst, S, lam, ubqp.DIVERSIFY, 3)
    check_round(Q, n, S, lam, orc.DIVERSIFY, 3, r, orc.first_derivative(Q))


@pytest.mark.parametrize("n", [2500, 5000, 6000])
def test_table1_sizes_eval(n):
    S = 1000
    Q = synth.make_instance(n, 1.0, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=n + 1)
    f = ubqp.eval(inst, X).cpu().numpy()
    Xh = orc.diversify(None, n, orc.RANDOM, n + 1, 0, S)
    assert np.array_equal(words_host(X), Xh)
    pick = np.array([0, 7, 500, 999])
    assert np.array_equal(f[pick], orc.eval(Q, Xh[pick]))
