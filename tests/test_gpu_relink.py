"""Path relinking (ubqp_relink) against the oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def host_words(t):
    return t.cpu().numpy().view(np.uint64)


def pairs_for(n, P, seed):
    """Random pairs plus the edge cases: equal solutions (distance 0), one
    differing bit (distance 1), near pairs (a few flips) and complements."""
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 2, (P, n)).astype(np.uint8)
    G = rng.integers(0, 2, (P, n)).astype(np.uint8)
    if P >= 5:
        G[0] = X[0]
        G[1] = X[1]
        G[1, rng.integers(0, n)] ^= 1
        G[2] = X[2]
        G[2, rng.choice(n, size=min(n, 3), replace=False)] ^= 1
        G[3] = 1 - X[3]
    return synth.pack_bits(X), synth.pack_bits(G)


@pytest.mark.parametrize("n", [1, 2, 5, 63, 64, 65, 100, 257, 300, 513, 1000, 1025, 2100, 4500])
@pytest.mark.parametrize("tensor_startup", [True, False])
def test_relink_matches_oracle(n, tensor_startup):
    Q = synth.make_instance(n, 0.5 if n > 64 else 1.0, n + 17)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    P = 12
    Xh, Gh = pairs_for(n, P, n)
    X = torch.from_numpy(Xh.view(np.int64)).cuda()
    G = torch.from_numpy(Gh.view(np.int64)).cuda()
    f = ubqp.eval(inst, X)
    Xb, fb, dist = ubqp.relink(inst, X, f, G, tensor_startup=tensor_startup)
    inst.sync()
    eXb, efb, ed = orc.relink(Q, Xh, Gh)
    assert np.array_equal(dist.cpu().numpy(), ed)
    assert np.array_equal(fb.cpu().numpy(), efb)
    assert np.array_equal(host_words(Xb), eXb)


def test_relink_full_size_sampled():
    """n = 7000 dense (the benchmark's instance): every pair's value is the
    oracle's objective of the returned solution; two pairs are replayed whole."""
    n = 7000
    Q = synth.make_instance(n, 1.0, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    P = 24
    Xh, Gh = pairs_for(n, P, 5)
    X = torch.from_numpy(Xh.view(np.int64)).cuda()
    G = torch.from_numpy(Gh.view(np.int64)).cuda()
    f = ubqp.eval(inst, X)
    Xb, fb, dist = ubqp.relink(inst, X, f, G)
    inst.sync()
    xb, fbh, dh = host_words(Xb), fb.cpu().numpy(), dist.cpu().numpy()
    assert np.array_equal(orc.eval(Q, xb), fbh)
    assert list(dh[:4]) == [0, 1, 3, n]
    for p in (2, 7):
        ex, ef, ed = orc.relink1(Q, Xh[p], Gh[p])
        assert (fbh[p], dh[p]) == (ef, ed) and np.array_equal(xb[p], ex)


def test_relink_rejects_small_workspace():
    Q = synth.make_instance(100, 0.5, 1)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    Xh, Gh = pairs_for(100, 8, 1)
    X = torch.from_numpy(Xh.view(np.int64)).cuda()
    G = torch.from_numpy(Gh.view(np.int64)).cuda()
    f = ubqp.eval(inst, X)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ubqp.UbqpError):
        ubqp.relink(inst, X, f, G, ws=small)


@pytest.mark.parametrize("n,extreme", [(9000, False), (2000, True)],
                         ids=["n9000_block512", "n2000_extreme_gains"])
def test_relink_large_and_extreme(n, extreme):
    """n = 9000 takes the 512-thread groups; |Q| = 127 dense makes the gains
    (positive and negative) as wide as the keys allow."""
    if extreme:
        rng = np.random.default_rng(3)
        Q = rng.choice(np.array([-127, 127], np.int8), size=(n, n))
        Q = np.triu(Q) + np.triu(Q, 1).T
    else:
        Q = synth.make_instance(n, 0.3, 90)
    inst = ubqp.Instance(torch.from_numpy(np.ascontiguousarray(Q)).cuda())
    P = 6
    Xh, Gh = pairs_for(n, P, n)
    X = torch.from_numpy(Xh.view(np.int64)).cuda()
    G = torch.from_numpy(Gh.view(np.int64)).cuda()
    f = ubqp.eval(inst, X, path=ubqp.EVAL_PLAIN)
    Xb, fb, dist = ubqp.relink(inst, X, f, G)
    inst.sync()
    for p in (1, 2, 4):
        ex, ef, ed = orc.relink1(Q, Xh[p], Gh[p])
        assert (int(fb[p].item()), int(dist[p].item())) == (ef, ed)
        assert np.array_equal(host_words(Xb)[p], ex)
