"""ubqp_ascent_trace on every group shape: the recorded flip sequence of each
climbed start equals the oracle's (orc_ascent1's trace), with a record
shorter than the climb (truncated, the climb itself unaffected), with a flip
cap, and for starts that are already local optima (nothing recorded)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def run(inst, X, f, idx, ldt, max_flips=0, sentinel=-7):
    S = X.shape[0]
    cnt = torch.tensor([idx.numel()], dtype=torch.int64, device="cuda")
    trace = torch.full((S, ldt), sentinel, dtype=torch.int16, device="cuda")
    flips, trace = ubqp.ascent_trace(inst, X, f, idx, cnt, ldt, max_flips=max_flips, trace=trace)
    inst.sync()
    return flips.cpu().numpy(), trace.cpu().numpy()


@pytest.mark.parametrize("n,density", [(40, 0.8), (300, 0.5), (700, 0.3), (1500, 1.0),
                                       (3000, 0.2), (9000, 0.1)])
def test_trace_equals_oracle_on_every_group_shape(n, density):
    # n <= 256 / 512: warp groups; 700: 64-thread blocks; 1500: 128; 3000: 256;
    # 9000: 512-thread blocks with two chunks
    Q = synth.make_instance(n, density, 17 + n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    S = 24 if n < 5000 else 6
    Xh = synth.random_solutions(n, S, n)
    X = torch.from_numpy(Xh.view(np.int64)).cuda()
    f0 = orc.eval(Q, Xh)
    f = torch.from_numpy(f0.copy()).cuda()
    idx = torch.arange(0, S, 2, dtype=torch.int32, device="cuda")  # every other start
    ldt = 2 * n
    flips, trace = run(inst, X, f, idx, ldt)
    for s in range(S):
        if s % 2:
            assert flips[s] == 0 and np.all(trace[s] == -7), s
            continue
        xw, fw, cw, tw = orc.ascent1(Q, Xh[s], int(f0[s]), 0, ldt)
        assert flips[s] == cw and int(f[s]) == fw, s
        assert np.array_equal(trace[s, :cw].view(np.uint16).astype(np.int64),
                              tw.astype(np.int64)), s
        assert np.all(trace[s, cw:] == -7), s   # entries past the climb untouched


def test_trace_truncated_and_capped():
    n, S = 1200, 8
    Q = synth.make_instance(n, 0.6, 5)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    Xh = synth.random_solutions(n, S, 5)
    f0 = orc.eval(Q, Xh)
    idx = torch.arange(S, dtype=torch.int32, device="cuda")
    # a record of 50 entries: the climbs run to their ends, the first 50 moves recorded
    X = torch.from_numpy(Xh.view(np.int64).copy()).cuda()
    f = torch.from_numpy(f0.copy()).cuda()
    flips, trace = run(inst, X, f, idx, 50)
    for s in range(S):
        xw, fw, cw, tw = orc.ascent1(Q, Xh[s], int(f0[s]), 0, 50)
        assert cw > 50 and flips[s] == cw and int(f[s]) == fw
        assert np.array_equal(X[s].cpu().numpy().view(np.uint64), xw)
        assert np.array_equal(trace[s].view(np.uint16).astype(np.int64), tw.astype(np.int64))
    # a flip cap of 17: 17 moves made and recorded
    X = torch.from_numpy(Xh.view(np.int64).copy()).cuda()
    f = torch.from_numpy(f0.copy()).cuda()
    flips, trace = run(inst, X, f, idx, 64, max_flips=17)
    for s in range(S):
        xw, fw, cw, tw = orc.ascent1(Q, Xh[s], int(f0[s]), 17, 64)
        assert cw == 17 and flips[s] == 17 and int(f[s]) == fw
        assert np.array_equal(trace[s, :17].view(np.uint16).astype(np.int64),
                              tw.astype(np.int64))
        assert np.all(trace[s, 17:] == -7)


def test_trace_of_local_optima_is_empty():
    n, S = 500, 6
    Q = synth.make_instance(n, 0.4, 8)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    Xh = synth.random_solutions(n, S, 8)
    f0 = orc.eval(Q, Xh)
    X = torch.from_numpy(Xh.view(np.int64).copy()).cuda()
    f = torch.from_numpy(f0.copy()).cuda()
    idx = torch.arange(S, dtype=torch.int32, device="cuda")
    run(inst, X, f, idx, n)           # climb once to local optima
    flips, trace = run(inst, X, f, idx, n)  # again: no move, nothing recorded
    assert np.all(flips == 0) and np.all(trace == -7)
