"""The ascent's launch for lists longer than the one-block-per-SM launch holds
(the fewest threads that hold n with two chunks each, several blocks per SM):
every group shape it uses (64 x 8 up to 256 x 2 blocks per SM), on lists far
above the capacity, against the same starts climbed in chunks small enough
for the one-block launch, and sampled starts -- those beyond the first waves
included -- against the oracle, flip sequence and all."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle_pool import OraclePool
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    p = OraclePool()
    yield p
    p.close()


@pytest.mark.parametrize("n", [1500, 2500, 3500, 4500, 5500, 6500, 8000])
def test_long_lists_equal_chunked_climbs_and_oracle(pool, n):
    S = 700
    Q = synth.make_instance(n, 0.7, 300 + n)
    ref = pool.put(Q)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X0 = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=n)
    f0 = ubqp.eval(inst, X0)
    ldt = 2 * n
    # the whole list at once: the several-blocks-per-SM launch
    X, f = X0.clone(), f0.clone()
    idx = torch.arange(S, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), S, dtype=torch.int64, device="cuda")
    flips, trace = ubqp.ascent_trace(inst, X, f, idx, cnt, ldt)
    # the same starts in chunks of 100 (a list the one-block launch holds)
    Xc, fc = X0.clone(), f0.clone()
    flc = torch.zeros(S, dtype=torch.int32, device="cuda")
    for a in range(0, S, 100):
        ic = torch.arange(a, min(a + 100, S), dtype=torch.int32, device="cuda")
        cc = torch.full((1,), ic.numel(), dtype=torch.int64, device="cuda")
        ubqp.ascent(inst, Xc, fc, ic, cc, 0, flc, ws=torch.empty(
            ubqp.ascent_workspace_size(inst, S), dtype=torch.uint8, device="cuda"))
    inst.sync()
    assert torch.equal(X, Xc) and torch.equal(f, fc) and torch.equal(flips, flc)
    # sampled starts against the oracle: first and last, and starts past the
    # first waves of both launches
    Xh = X0.cpu().numpy().view(np.uint64)
    fh = f0.cpu().numpy()
    pick = sorted({0, 1, 151, 152, 153, 455, 456, 457, S - 2, S - 1} |
                  set(np.random.default_rng(n).integers(0, S, 10).tolist()))
    want = pool.ascents(ref, Xh, fh, pick, cap=ldt)
    Xg, fg, flg = X.cpu().numpy().view(np.uint64), f.cpu().numpy(), flips.cpu().numpy()
    tr = trace.cpu().numpy().view(np.uint16)
    for s in pick:
        xw, fw, cw, tw = want[s]
        assert int(fg[s]) == fw and int(flg[s]) == cw and np.array_equal(Xg[s], xw), s
        assert np.array_equal(tr[s, :cw].astype(np.int64), tw.astype(np.int64)), s
