"""Bit-exact parity of every CUDA step with the CPU oracle, through the C ABI.

All inputs are seeded and synthetic (paper_1706_00037_gb300.synth); no oracle
input comes from the CUDA path.  Integer results (objective values, indices,
solutions, flip counts) must be identical; the screening threshold is compared
for exact equality too, since both sides evaluate the same rounded operations.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu

NS = [1, 2, 3, 63, 64, 65, 100, 127, 128, 129, 257, 511, 512, 513, 1000, 1025, 2100]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def words_dev(X):
    return dev(np.ascontiguousarray(X, dtype=np.uint64).view(np.int64))


def words_host(t):
    return t.cpu().numpy().view(np.uint64)


def instance(n, density, seed, ldq=None):
    Q = synth.make_instance(n, density, seed, ldq=ldq)
    return Q, ubqp.Instance(dev(Q))


# ----------------------------------------------------------------- prepare

@pytest.mark.parametrize("n", NS)
def test_prepare_first_derivative(n):
    Q, inst = instance(n, 0.3, n)
    assert inst.n == n and inst.words == synth.words(n)
    assert inst.max_abs == int(np.abs(Q.astype(np.int32)).max())
    x0 = ubqp.first_derivative(inst)
    assert np.array_equal(words_host(x0), orc.first_derivative(Q))


def test_prepare_rejects_asymmetric():
    Q = synth.make_instance(70, 0.5, 1)
    Q[3, 60] = Q[60, 3] + 1
    with pytest.raises(ubqp.UbqpError) as e:
        ubqp.Instance(dev(Q))
    assert e.value.status == -2


def test_prepare_ignores_bytes_beyond_n():
    n, ldq = 77, 128
    Q = synth.make_instance(n, 0.5, 5, ldq=ldq)
    Q[:, n:] = 55  # asymmetric garbage outside the instance
    inst = ubqp.Instance(dev(Q))
    X = synth.random_solutions(n, 20, 1)
    f = ubqp.eval(inst, words_dev(X), path=ubqp.EVAL_PLAIN)
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


# ----------------------------------------------------------------- diversify

@pytest.mark.parametrize("n", [1, 5, 64, 65, 100, 130, 1000])
@pytest.mark.parametrize("mode", [orc.RANDOM, orc.DIVERSIFY])
def test_diversify_matches_oracle(n, mode):
    Q, inst = instance(n, 0.2, 3)
    S = 301
    for round_, div_H, seed in ((0, 64, 7), (3, 5, 2**63 + 11)):
        X = ubqp.diversify(inst, S, mode=mode, seed=seed, round_=round_, div_H=div_H)
        want = orc.diversify(orc.first_derivative(Q), n, mode, seed, round_, S, div_H)
        assert np.array_equal(words_host(X), want)


def test_diversify_explicit_incumbent():
    n, S = 200, 64
    Q, inst = instance(n, 0.2, 4)
    x0 = synth.random_solutions(n, 1, 9)[0]
    X = ubqp.diversify(inst, S, mode=orc.DIVERSIFY, seed=5, x0=words_dev(x0))
    assert np.array_equal(words_host(X), orc.diversify(x0, n, orc.DIVERSIFY, 5, 0, S))


# ----------------------------------------------------------------- eval

@pytest.mark.parametrize("n", NS)
def test_eval_plain_matches_oracle(n):
    Q, inst = instance(n, 0.6, n + 100)
    X = synth.random_solutions(n, 37, n)
    f = ubqp.eval(inst, words_dev(X), path=ubqp.EVAL_PLAIN)
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


TC_PATHS = [ubqp.EVAL_TC, ubqp.EVAL_TC_TMEM]


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("S", [1, 37, 129, 300])
@pytest.mark.parametrize("path", TC_PATHS)
def test_eval_tc_matches_oracle(n, S, path):
    Q, inst = instance(n, 0.6, n + 200)
    X = synth.random_solutions(n, S, n + S)
    f = ubqp.eval(inst, words_dev(X), path=path)
    inst.sync()
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


@pytest.mark.parametrize("path", TC_PATHS + [ubqp.EVAL_TC_STAGED])
def test_eval_tc_extreme_coefficients_exact(path):
    # |Q| at the int8 limits and dense 0/1 patterns: every fp32 partial stays an
    # exact integer only if the chunked accumulation is right
    n = 1500
    Q = np.full((n, n), -128, np.int8)
    np.fill_diagonal(Q, 127)
    Q[:700, :700] = 127
    inst = ubqp.Instance(dev(Q))
    X = np.concatenate([synth.random_solutions(n, 60, 5), synth.random_solutions(n, 60, 6, 0.95),
                        synth.pack_bits(np.ones((4, n), np.uint8)),
                        np.zeros((1, synth.words(n)), np.uint64)])
    f = ubqp.eval(inst, words_dev(X), path=path)
    inst.sync()
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


@pytest.mark.parametrize("n,S", [(2500, 1000), (5000, 1000)])
def test_eval_tc_equals_plain_at_table1_sizes(n, S):
    Q, inst = instance(n, 1.0, n)
    X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=n + 1)
    ft = ubqp.eval(inst, X, path=ubqp.EVAL_TC)
    fp = ubqp.eval(inst, X, path=ubqp.EVAL_PLAIN)
    fm = ubqp.eval(inst, X, path=ubqp.EVAL_TC_TMEM)
    inst.sync()
    assert torch.equal(ft, fp) and torch.equal(fm, fp)
    # sampled starts against the oracle (its inputs regenerated on the CPU)
    Xh = orc.diversify(None, n, orc.RANDOM, n + 1, 0, S)
    pick = np.array([0, 1, S // 2, S - 1])
    assert np.array_equal(ft.cpu().numpy()[pick], orc.eval(Q, Xh[pick]))


def test_eval_tc_workspace_errors():
    n, S = 300, 50
    Q, inst = instance(n, 0.5, 1)
    X = words_dev(synth.random_solutions(n, S, 1))
    need = ubqp.eval_workspace_size(inst, S, ubqp.EVAL_TC_STAGED)
    assert need == 128 * 512 * 2
    small = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ubqp.UbqpError) as e:
        ubqp.eval(inst, X, path=ubqp.EVAL_TC_STAGED, ws=small)
    assert e.value.status == -4
    assert ubqp.eval_workspace_size(inst, S, ubqp.EVAL_PLAIN) == 0
    assert ubqp.eval_workspace_size(inst, S, ubqp.EVAL_TC) == 0
    assert ubqp.eval_workspace_size(inst, S, ubqp.EVAL_TC_TMEM) == 0


@pytest.mark.parametrize("n,S,fused", [(300, 50, False), (300, 4095, False), (300, 4096, True),
                                       (1024, 8192, True), (1025, 8192, False),
                                       (7000, 1000, False)])
def test_eval_auto_path_choice(n, S, fused):
    # AUTO takes the fused operand build (no workspace) only for n padded to
    # at most 1024 with at least 4096 starts, the staged one otherwise; the
    # values agree either way
    Q, inst = instance(n, 0.5, 3)
    need = ubqp.eval_workspace_size(inst, S, ubqp.EVAL_AUTO)
    assert need == (0 if fused else ubqp.eval_workspace_size(inst, S, ubqp.EVAL_TC_STAGED))
    X = words_dev(synth.random_solutions(n, S, 4))
    f_auto = ubqp.eval(inst, X, path=ubqp.EVAL_AUTO)
    f_other = ubqp.eval(inst, X, path=ubqp.EVAL_TC_STAGED if fused else ubqp.EVAL_TC)
    assert torch.equal(f_auto, f_other)
    pick = np.arange(0, S, max(1, S // 7))
    Xh = synth.random_solutions(n, S, 4)
    assert np.array_equal(f_auto.cpu().numpy()[pick], orc.eval(Q, Xh[pick]))


@pytest.mark.parametrize("n", [1, 65, 257, 1000, 2100])
@pytest.mark.parametrize("S", [1, 129, 300])
def test_eval_tc_staged_matches_oracle(n, S):
    Q, inst = instance(n, 0.6, n + 300)
    X = synth.random_solutions(n, S, n + 2 * S)
    f = ubqp.eval(inst, words_dev(X), path=ubqp.EVAL_TC_STAGED)
    inst.sync()
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


def test_eval_ignores_pad_bits():
    n = 70
    Q, inst = instance(n, 1.0, 2)
    X = synth.random_solutions(n, 9, 2)
    Xd = X.copy()
    Xd[:, -1] |= np.uint64(0xFFFF) << np.uint64(48)  # set bits >= n
    for path in (ubqp.EVAL_PLAIN, ubqp.EVAL_TC, ubqp.EVAL_TC_STAGED, ubqp.EVAL_TC_TMEM):
        f = ubqp.eval(inst, words_dev(Xd), path=path)
        assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


def test_eval_extreme_coefficients():
    n = 300
    Q = np.full((n, n), -128, np.int8)
    np.fill_diagonal(Q, 127)
    inst = ubqp.Instance(dev(Q))
    X = np.concatenate([synth.random_solutions(n, 6, 1),
                        synth.pack_bits(np.ones((1, n), np.uint8)),
                        np.zeros((1, synth.words(n)), np.uint64)])
    f = ubqp.eval(inst, words_dev(X), path=ubqp.EVAL_PLAIN)
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X))


# ----------------------------------------------------------------- screen

@pytest.mark.parametrize("S", [1, 2, 1023, 1024, 1025, 8192, 20000])
@pytest.mark.parametrize("lam", [0.0, 0.25, 0.5, 0.75, 1.0])
def test_screen_matches_oracle(S, lam):
    r = np.random.default_rng(S)
    fv = r.integers(-5 * 10**9, 5 * 10**9, S).astype(np.int64)
    fv[r.integers(0, S, max(1, S // 10))] = fv.max()  # ties at the max
    out = ubqp.screen(dev(fv), lam)
    want = orc.screen(fv, lam)
    c = int(out["count"].item())
    assert c == want["count"]
    assert np.array_equal(out["idx"][:c].cpu().numpy(), want["idx"])
    Tm = out["Tm"].cpu().numpy()
    assert Tm[0] == want["T"] and Tm[1] == want["mean"]
    assert list(out["stats"].cpu().numpy()) == [want["sum"], want["max"], want["argmax"]]


def test_screen_all_equal_and_threshold_ties():
    fv = np.full(777, 42, np.int64)
    out = ubqp.screen(dev(fv), 0.5)
    assert int(out["count"].item()) == 0
    fv = np.array([0, 9, 12, 3], np.int64)  # T = 9 exactly; 9 does not pass
    out = ubqp.screen(dev(fv), 0.5)
    assert int(out["count"].item()) == 1 and int(out["idx"][0].item()) == 2


# ----------------------------------------------------------------- ascent

def _ascent_case(n, density, seed, S, max_flips=0, idx=None, use_ws=True):
    Q, inst = instance(n, density, seed)
    X = synth.random_solutions(n, S, seed + 1)
    fv = orc.eval(Q, X)
    idx = np.arange(S, dtype=np.int32) if idx is None else np.asarray(idx, np.int32)
    Xd, fd = words_dev(X), dev(fv)
    flips = torch.full((S,), -1, dtype=torch.int32, device="cuda")
    ubqp.ascent(inst, Xd, fd, dev(idx), dev(np.array([len(idx)], np.int64)), max_flips, flips,
                use_ws=use_ws)
    inst.sync()
    Xw, fw, flw = orc.ascent(Q, X, fv, idx, max_flips)
    flw = np.where(np.isin(np.arange(S), idx), flw, -1)
    return words_host(Xd), fd.cpu().numpy(), flips.cpu().numpy(), Xw, fw, flw


@pytest.mark.parametrize("use_ws", [True, False], ids=["tc_startup", "core_startup"])
@pytest.mark.parametrize("n", NS)
def test_ascent_matches_oracle(n, use_ws):
    Xg, fg, flg, Xw, fw, flw = _ascent_case(n, 0.5, n + 7, 24, use_ws=use_ws)
    assert np.array_equal(fg, fw)
    assert np.array_equal(flg, flw)
    assert np.array_equal(Xg, Xw)


@pytest.mark.parametrize("n,density", [(100, 0.1), (700, 1.0), (3000, 0.1)])
def test_ascent_subset_and_untouched(n, density):
    S = 40
    idx = [3, 0, 17, 39, 22]
    for use_ws in (True, False):
        Xg, fg, flg, Xw, fw, flw = _ascent_case(n, density, 11, S, idx=idx, use_ws=use_ws)
        assert np.array_equal(fg, fw) and np.array_equal(flg, flw) and np.array_equal(Xg, Xw)


@pytest.mark.parametrize("n,extreme", [(8192, True), (9000, False)],
                         ids=["n8192_wide_gains", "n9000_block512"])
def test_ascent_large_n_paths(n, extreme):
    # n = 8192 with |Q| = 128 exceeds the packed-key gain bound (two-step warp
    # reduction); n = 9000 takes the 512-thread groups
    S = 3
    if extreme:
        r = np.random.default_rng(1)
        Q = np.where(r.random((n, n)) < 0.5, 127, -128).astype(np.int8)
        Q = np.triu(Q) + np.triu(Q, 1).T
    else:
        Q = synth.make_instance(n, 0.5, 9)
    inst = ubqp.Instance(dev(Q))
    X = synth.random_solutions(n, S, 4)
    fv = orc.eval(Q, X)
    for use_ws in (True, False):
        Xd, fd = words_dev(X), dev(fv)
        flips = torch.zeros(S, dtype=torch.int32, device="cuda")
        ubqp.ascent(inst, Xd, fd, dev(np.arange(S, dtype=np.int32)),
                    dev(np.array([S], np.int64)), 0, flips, use_ws=use_ws)
        inst.sync()
        if use_ws:
            Xw, fw, flw = orc.ascent(Q, X, fv, np.arange(S, dtype=np.int32))
        assert np.array_equal(fd.cpu().numpy(), fw)
        assert np.array_equal(flips.cpu().numpy(), flw)
        assert np.array_equal(words_host(Xd), Xw)


@pytest.mark.parametrize("n,S", [(200, 20000), (700, 3000)],
                         ids=["warp_groups", "block64_groups"])
def test_ascent_more_starts_than_the_first_wave(n, S):
    """Every start climbed, many more than the persistent groups (four warps
    per block at n = 200, 64-thread blocks at n = 700): the starts beyond the
    first wave come from the workspace's counter, each exactly once, and every
    value, flip count and solution equals the oracle's."""
    Q = synth.make_instance(n, 0.5, n + 1)
    inst = ubqp.Instance(dev(Q))
    X = synth.random_solutions(n, S, 5)
    fv = orc.eval(Q, X)
    Xw, fw, flw = orc.ascent(Q, X, fv, np.arange(S, dtype=np.int32))
    Xd, fd = words_dev(X), dev(fv)
    flips = torch.zeros(S, dtype=torch.int32, device="cuda")
    ubqp.ascent(inst, Xd, fd, dev(np.arange(S, dtype=np.int32)), dev(np.array([S], np.int64)),
                0, flips, use_ws=True)
    inst.sync()
    assert np.array_equal(flips.cpu().numpy(), flw)
    assert np.array_equal(fd.cpu().numpy(), fw)
    assert np.array_equal(words_host(Xd), Xw)


def test_ascent_startup_extreme_coefficients():
    # |Q| at the int8 limits: the tensor-core start-up y = Q x must stay exact
    n, S = 1200, 30
    Q = np.full((n, n), -128, np.int8)
    np.fill_diagonal(Q, 127)
    Q[:500, :500] = 127
    inst = ubqp.Instance(dev(Q))
    X = np.concatenate([synth.random_solutions(n, S - 2, 3, 0.9),
                        synth.pack_bits(np.ones((1, n), np.uint8)),
                        np.zeros((1, synth.words(n)), np.uint64)])
    fv = orc.eval(Q, X)
    Xd, fd = words_dev(X), dev(fv)
    flips = torch.zeros(S, dtype=torch.int32, device="cuda")
    ubqp.ascent(inst, Xd, fd, dev(np.arange(S, dtype=np.int32)), dev(np.array([S], np.int64)),
                0, flips)
    inst.sync()
    Xw, fw, flw = orc.ascent(Q, X, fv, np.arange(S, dtype=np.int32))
    assert np.array_equal(fd.cpu().numpy(), fw) and np.array_equal(flips.cpu().numpy(), flw)
    assert np.array_equal(words_host(Xd), Xw)


@pytest.mark.parametrize("n", [50, 600])
def test_ascent_flip_sequence_prefixes(n):
    # capping the flips at m must give the first m moves of the uncapped run
    Q, inst = instance(n, 1.0, 21)
    x = synth.random_solutions(n, 1, 21)
    f0 = orc.eval(Q, x)
    _, _, full, trace = orc.ascent1(Q, x[0], int(f0[0]), trace_cap=10**6)
    assert full >= 5
    for m in (1, 2, 3, full // 2, full, full + 3):
        Xd, fd = words_dev(x), dev(f0)
        flips = torch.zeros(1, dtype=torch.int32, device="cuda")
        ubqp.ascent(inst, Xd, fd, dev(np.zeros(1, np.int32)), dev(np.ones(1, np.int64)), m,
                    flips)
        xw, fw, cw, _ = orc.ascent1(Q, x[0], int(f0[0]), max_flips=m)
        assert int(flips.item()) == cw == min(m, full)
        assert np.array_equal(words_host(Xd)[0], xw) and int(fd.item()) == fw
        # the flipped set is exactly the first m indices of the trace
        diff = synth.unpack_bits(words_host(Xd)[0] ^ x[0], n)
        odd = np.zeros(n, np.int64)
        for k in trace[:min(m, full)]:
            odd[k] ^= 1
        assert np.array_equal(diff, odd)


def test_ascent_empty_and_degenerate():
    n = 90
    Q = np.zeros((n, n), np.int8)  # every gain is 0: nothing improves
    inst = ubqp.Instance(dev(Q))
    X = synth.random_solutions(n, 5, 1)
    Xd, fd = words_dev(X), dev(np.zeros(5, np.int64))
    flips = torch.zeros(5, dtype=torch.int32, device="cuda")
    ubqp.ascent(inst, Xd, fd, dev(np.arange(5, dtype=np.int32)), dev(np.array([5], np.int64)),
                0, flips)
    assert np.array_equal(words_host(Xd), X) and flips.sum().item() == 0
    # count = 0: nothing runs
    ubqp.ascent(inst, Xd, fd, dev(np.arange(5, dtype=np.int32)), dev(np.array([0], np.int64)),
                0, flips)
    inst.sync()
    # single variable with positive diagonal: one flip from 0
    Q1 = np.array([[7]], np.int8)
    inst1 = ubqp.Instance(dev(Q1))
    Xd = words_dev(np.zeros((1, 1), np.uint64))
    fd = dev(np.zeros(1, np.int64))
    ubqp.ascent(inst1, Xd, fd, dev(np.zeros(1, np.int32)), dev(np.ones(1, np.int64)), 0, None)
    assert int(words_host(Xd)[0, 0]) == 1 and int(fd.item()) == 7


# ----------------------------------------------------------------- best / solve

def test_best_matches_oracle():
    fv = np.array([5, 9, -1, 9, 3], np.int64)
    X = synth.random_solutions(40, 5, 3)
    bx, bf = ubqp.best(dev(fv), words_dev(X))
    assert list(bf.cpu().numpy()) == [9, 1]
    assert np.array_equal(words_host(bx), X[1])


@pytest.mark.parametrize("path", [ubqp.EVAL_TC, ubqp.EVAL_PLAIN])
@pytest.mark.parametrize("mode", [orc.DIVERSIFY, orc.RANDOM])
def test_solve_small_instance_matches_oracle(mode, path):
    # n = 100, density 0.1 (diagonal included), seed 0; 1000 starts, lambda 0.5
    n, S, lam = 100, 1000, 0.5
    Q, inst = instance(n, 0.1, 0)
    p = ubqp.make_params(S, lam, mode=mode, seed=0, eval_path=path)
    bx, bf, st = ubqp.solve(inst, p)
    want = orc.solve(Q, S, lam, seed=0, mode=mode)
    assert int(bf[0].item()) == want["best_f"] and int(bf[1].item()) == want["best_index"]
    assert np.array_equal(words_host(bx), want["best_x"])
    for k in ("passed", "total_flips", "max_flips_seen", "batch_max", "best_index", "sum",
              "T", "mean"):
        assert st[k] == want[k], k


@pytest.mark.parametrize("lam", [0.25, 0.5, 0.75])
def test_solve_pipeline_steps_match_oracle(lam):
    n, S = 300, 500
    Q, inst = instance(n, 0.1, 3)
    x0 = orc.first_derivative(Q)
    X = orc.diversify(x0, n, orc.DIVERSIFY, 3, 0, S)
    fv = orc.eval(Q, X)
    sc = orc.screen(fv, lam)
    Xw, fw, _ = orc.ascent(Q, X, fv, sc["idx"])
    bw = orc.best(fw)
    p = ubqp.make_params(S, lam, seed=3)
    bx, bf, st = ubqp.solve(inst, p)
    assert st["passed"] == sc["count"] and st["T"] == sc["T"]
    assert (int(bf[0].item()), int(bf[1].item())) == bw
    assert np.array_equal(words_host(bx), Xw[bw[1]])


def test_instance_in_caller_arena_solves_identically():
    n = 777
    Q = synth.make_instance(n, 0.4, 31)
    arena = torch.empty(ubqp.arena_size(n), dtype=torch.uint8, device="cuda")
    a = ubqp.Instance(dev(Q))
    b = ubqp.Instance(dev(Q), arena=arena)
    p = ubqp.make_params(500, 0.5, seed=9)
    xa, fa, sa = ubqp.solve(a, p)
    xb, fb, sb = ubqp.solve(b, p)
    assert torch.equal(xa, xb) and torch.equal(fa, fb) and sa == sb
    small = torch.empty(ubqp.arena_size(n) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ubqp.UbqpError):
        ubqp.Instance(dev(Q), arena=small)


def test_instance_from_pinned_host_memory_solves_identically():
    """Q in page-locked host memory is read in place by the preparing kernel:
    the same instance (max |Q|, first-derivative start, solve) as from a device
    copy, with and without an arena; asymmetry is still caught; pageable host
    memory is refused by the library itself."""
    import ctypes
    n, ldq = 777, 800
    Q = synth.make_instance(n, 0.4, 31, ldq=ldq)
    a = ubqp.Instance(dev(Q))
    pinned = torch.from_numpy(Q).pin_memory()
    arena = torch.empty(ubqp.arena_size(n), dtype=torch.uint8, device="cuda")
    p = ubqp.make_params(500, 0.5, seed=9)
    xa, fa, sa = ubqp.solve(a, p)
    for b in (ubqp.Instance(pinned), ubqp.Instance(pinned, arena=arena)):
        assert b.max_abs == a.max_abs
        assert torch.equal(ubqp.first_derivative(b), ubqp.first_derivative(a))
        xb, fb, sb = ubqp.solve(b, p)
        assert torch.equal(xa, xb) and torch.equal(fa, fb) and sa == sb
    bad = Q.copy()
    bad[3, 60] = bad[60, 3] + 1
    with pytest.raises(ubqp.UbqpError) as e:
        ubqp.Instance(torch.from_numpy(bad).pin_memory())
    assert e.value.status == -2
    pageable = np.ascontiguousarray(Q)
    h = ctypes.c_void_p()
    assert ubqp.load().ubqp_q_prepare(pageable.ctypes.data_as(ctypes.c_void_p), n, ldq, None,
                                      ctypes.byref(h)) == -1
    assert not h.value


def test_deferred_validation_instance():
    """ubqp_q_prepare_into_async: the same instance without a synchronisation;
    the first sync reports the symmetry check and max |Q|, and every later sync
    keeps reporting an asymmetric Q."""
    n = 777
    Q = synth.make_instance(n, 0.4, 31)
    a = ubqp.Instance(dev(Q))
    arena = torch.empty(ubqp.arena_size(n), dtype=torch.uint8, device="cuda")
    Qd = dev(Q)  # must live until the preparation has run
    b = ubqp.Instance(Qd, arena=arena, defer_validation=True)
    assert b.max_abs == -1
    p = ubqp.make_params(500, 0.5, seed=9)
    xa, fa, sa = ubqp.solve(a, p)
    xb, fb, sb = ubqp.solve(b, p)
    b.sync()
    assert b.max_abs == a.max_abs
    assert torch.equal(xa, xb) and torch.equal(fa, fb) and sa == sb
    b.close()
    bad = Q.copy()
    bad[3, 60] = bad[60, 3] + 1
    Qbad = dev(bad)
    c = ubqp.Instance(Qbad, arena=arena, defer_validation=True)
    for _ in range(2):
        with pytest.raises(ubqp.UbqpError) as e:
            c.sync()
        assert e.value.status == -2
    c.close()
    with pytest.raises(ValueError):
        ubqp.Instance(Qd, defer_validation=True)  # needs an arena


@pytest.mark.parametrize("path", [ubqp.EVAL_PLAIN, ubqp.EVAL_TC, ubqp.EVAL_TC_STAGED,
                                  ubqp.EVAL_TC_TMEM])
def test_eval_all_solutions_of_a_small_instance(path):
    """Every one of the 2^14 solutions: the evaluation against a numpy product,
    its maximum and first maximiser against the oracle's exhaustive search."""
    n = 14
    Q = synth.make_instance(n, 0.8, 77)
    inst = ubqp.Instance(dev(Q))
    k = np.arange(2 ** n, dtype=np.uint64)
    X = k.reshape(-1, 1)  # solution number = its bit pattern, one word each
    f = ubqp.eval(inst, words_dev(X), path=path).cpu().numpy()
    bits = ((k[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
    Qn = Q[:, :n].astype(np.int64)
    assert np.array_equal(f, np.einsum("si,ij,sj->s", bits, Qn, bits))
    gmax, gx = orc.brute_force(Q)
    assert f.max() == gmax and int(np.argmax(f)) == gx
