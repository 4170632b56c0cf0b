"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks one oracle function against the mathematics or a hand-worked
case: closed forms of problem (P), brute force on instances with a known
optimum (max-cut, a UBQP application the paper lists), the 1-flip move value
recomputed from f itself, and hand-worked screening and diversification
cases.  None of them retypes the oracle's own formula.
"""
import os

import numpy as np
import pytest

import oracle as orc
from paper_1706_00037_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f_np(Q, x01):
    """Independent evaluation with a numpy int64 matrix product."""
    x = np.asarray(x01, dtype=np.int64)
    Qn = np.asarray(Q[:, :Q.shape[0]], dtype=np.int64)
    return int(x @ Qn @ x)


# ---------------------------------------------------------------- SplitMix64

def test_splitmix64_published_vector():
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = [int(l) for l in lines[1:]]
    g = 0x9E3779B97F4A7C15
    got = [orc.splitmix64((seed + k * g) % 2**64) for k in range(len(expect))]
    assert got == expect


def test_synth_rng_matches_published_vector():
    # the instance generator's own SplitMix64 (a separate implementation)
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = [int(l) for l in lines[1:]]
    g = 0x9E3779B97F4A7C15
    ctr = np.array([(seed + k * g) % 2**64 for k in range(len(expect))], np.uint64)
    got = synth.rng_array(0, 0, ctr)
    assert [int(v) for v in got] == expect


# ---------------------------------------------------------------- objective

@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 1), (7, 0.5, 2), (64, 0.1, 3),
                                            (65, 1.0, 4), (130, 0.3, 5)])
def test_f_closed_forms(n, density, seed):
    Q = synth.make_instance(n, density, seed)
    W = synth.words(n)
    zero = np.zeros(W, np.uint64)
    assert orc.f(Q, zero) == 0
    ones = synth.pack_bits(np.ones(n, np.uint8))
    assert orc.f(Q, ones) == int(Q.astype(np.int64).sum())
    r = np.random.default_rng(seed)
    for _ in range(5):
        i, j = r.integers(0, n, 2)
        e = np.zeros(n, np.uint8)
        e[i] = 1
        assert orc.f(Q, synth.pack_bits(e)) == int(Q[i, i])
        if i != j:
            e[j] = 1
            assert orc.f(Q, synth.pack_bits(e)) == int(Q[i, i]) + int(Q[j, j]) + 2 * int(Q[i, j])


@pytest.mark.parametrize("n", [3, 63, 64, 65, 129, 200])
def test_f_matches_matrix_product(n):
    Q = synth.make_instance(n, 0.7, n)
    X01 = (np.random.default_rng(n).random((8, n)) < 0.5).astype(np.uint8)
    X = synth.pack_bits(X01)
    got = orc.eval(Q, X)
    want = [_f_np(Q, x) for x in X01]
    assert list(got) == want


def test_f_respects_row_stride():
    n, ldq = 37, 64
    Q = synth.make_instance(n, 0.8, 11, ldq=ldq)
    Q[:, n:] = 99  # bytes beyond column n are not part of the instance
    X01 = (np.random.default_rng(1).random((4, n)) < 0.5).astype(np.uint8)
    assert list(orc.eval(Q, synth.pack_bits(X01))) == [_f_np(Q, x) for x in X01]


def _maxcut_graphs():
    out = []
    for line in open(os.path.join(GOLDEN, "maxcut_graphs.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        head, edges = line.split("|")
        name, n, opt = head.split()
        E = [tuple(int(t) for t in e.split("-")) for e in edges.split()]
        out.append((name, int(n), int(opt), E))
    return out


def _maxcut_q(n, E):
    Q = np.zeros((n, n), np.int8)
    for a, b in E:
        Q[a, b] -= 1
        Q[b, a] -= 1
        Q[a, a] += 1
        Q[b, b] += 1
    return Q


@pytest.mark.parametrize("g", _maxcut_graphs(), ids=lambda g: g[0])
def test_brute_force_maxcut_optimum(g):
    name, n, opt, E = g
    Q = _maxcut_q(n, E)
    best, bits = orc.brute_force(Q)
    assert best == opt
    x01 = [(bits >> j) & 1 for j in range(n)]
    cut = sum(1 for a, b in E if x01[a] != x01[b])
    assert cut == opt


@pytest.mark.parametrize("g", _maxcut_graphs(), ids=lambda g: g[0])
def test_ascent_on_maxcut_is_local_and_bounded(g):
    name, n, opt, E = g
    Q = _maxcut_q(n, E)
    for seed in range(4):
        x = synth.random_solutions(n, 1, seed)[0]
        f0 = _f_np(Q, synth.unpack_bits(x, n))
        xn, fn, flips, _ = orc.ascent1(Q, x, f0)
        assert fn <= opt
        assert fn == _f_np(Q, synth.unpack_bits(xn, n))
        # local optimum: no single flip improves
        x01 = synth.unpack_bits(xn, n).astype(np.int64)
        for i in range(n):
            y = x01.copy()
            y[i] ^= 1
            assert _f_np(Q, y) <= fn


# ---------------------------------------------------------------- first derivative

def test_first_derivative_rowsum_sign():
    n = 70
    Q = synth.make_instance(n, 0.2, 7)
    # force one row sum to exactly zero (keep symmetry): row/col 5 -> 0
    Q[5, :] = 0
    Q[:, 5] = 0
    rs = Q.astype(np.int64).sum(axis=1)
    assert rs[5] == 0
    x0 = orc.first_derivative(Q)
    got = synth.unpack_bits(x0, n)
    assert list(got) == [1 if r > 0 else 0 for r in rs]
    assert x0[-1] >> np.uint64(n - 64) == 0  # pad bits clear


# ---------------------------------------------------------------- diversify

def test_diversify_random_mode_words_and_padding():
    n, S, seed = 100, 5, 42
    X = orc.diversify(None, n, orc.RANDOM, seed, 0, S)
    g = 0x9E3779B97F4A7C15
    for s in range(S):
        for w in range(2):
            raw = orc.splitmix64(seed ^ ((s * g) % 2**64) ^ w)
            if w == 1:
                raw &= (1 << (n - 64)) - 1
            assert int(X[s, w]) == raw


def test_diversify_hpattern_hand_cases():
    n, S = 10, 12
    X = orc.diversify(np.zeros(1, np.uint64), n, orc.DIVERSIFY, 5, 0, S, div_H=3)
    for line in open(os.path.join(GOLDEN, "diversify_hpattern.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        i, bits = line.split("|")
        i = int(i)
        want = sum(1 << int(b) for b in bits.split())
        assert int(X[i, 0]) == want, i


def test_diversify_hpattern_is_relative_to_incumbent():
    n, S = 150, 40
    x0 = synth.random_solutions(n, 1, 3)[0]
    Xz = orc.diversify(np.zeros_like(x0), n, orc.DIVERSIFY, 9, 0, S)
    Xi = orc.diversify(x0, n, orc.DIVERSIFY, 9, 0, S)
    for i in range(0, S, 2):  # even counters: a fixed flip pattern xor-ed in
        assert np.array_equal(Xi[i], Xz[i] ^ x0)
    assert np.array_equal(Xi[0], x0)


def test_diversify_breed_is_a_masked_blend():
    # odd counters blend the incumbent with a partner through a mask that does
    # not depend on the incumbent: child = (x0 & ~mask) | (partner & mask).
    # With x0 = 0 the child is partner & mask; with x0 = 1 it is ~mask | partner.
    n, S = 200, 1200
    ones = synth.pack_bits(np.ones(n, np.uint8))
    x0 = synth.random_solutions(n, 1, 4)[0]
    X = orc.diversify(x0, n, orc.DIVERSIFY, 77, 0, S)
    X1 = orc.diversify(ones, n, orc.DIVERSIFY, 77, 0, S)
    X0 = orc.diversify(np.zeros_like(x0), n, orc.DIVERSIFY, 77, 0, S)
    frac = {m: [] for m in range(1, 7)}
    for i in range(1, S, 2):
        mask = ~(X0[i] ^ X1[i]) & ones
        assert np.array_equal(X0[i] & ~mask, np.zeros_like(x0))
        assert np.array_equal(X[i], (x0 & ~mask) | X0[i])
        m = 1 + ((i - 1) // 2) % 6
        frac[m].append(sum(bin(int(w)).count("1") for w in mask) / n)
    # each bit comes from the partner with probability 2^-m
    for m, v in frac.items():
        assert abs(np.mean(v) - 2.0 ** -m) < 0.02, (m, np.mean(v))


def test_diversify_round_counter_continues():
    n, S = 90, 8
    x0 = synth.random_solutions(n, 1, 8)[0]
    big = orc.diversify(x0, n, orc.DIVERSIFY, 3, 0, 2 * S)
    r1 = orc.diversify(x0, n, orc.DIVERSIFY, 3, 1, S)
    # the starts of the second search round (round index 1, S per round) are the
    # loop counters S..2S-1
    assert np.array_equal(r1, big[S:])


# ---------------------------------------------------------------- screen

def _screen_cases():
    out = []
    for line in open(os.path.join(GOLDEN, "screen_cases.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        lam, fv, idx, T, mean, mx, am = [p.strip() for p in line.split("|")]
        out.append((float(lam), [int(v) for v in fv.split()], [int(v) for v in idx.split()],
                    float(T), float(mean), int(mx), int(am)))
    return out


@pytest.mark.parametrize("case", _screen_cases())
def test_screen_hand_cases(case):
    lam, fv, idx, T, mean, mx, am = case
    r = orc.screen(np.array(fv, np.int64), lam)
    assert list(r["idx"]) == idx
    assert r["T"] == T and r["mean"] == mean and r["max"] == mx and r["argmax"] == am
    assert list(np.nonzero(orc.screen_exact(np.array(fv, np.int64), lam))[0]) == idx


@pytest.mark.parametrize("lam", [0.0, 0.25, 0.5, 0.75, 1.0])
def test_screen_fp64_agrees_with_exact_rational(lam):
    r = np.random.default_rng(int(lam * 100))
    for scale in (10, 10**6, 4 * 10**9):
        fv = r.integers(-scale, scale, 5000).astype(np.int64)
        got = np.zeros(fv.shape[0], bool)
        got[orc.screen(fv, lam)["idx"]] = True
        assert np.array_equal(got, orc.screen_exact(fv, lam))


def test_screen_special_cases():
    fv = np.random.default_rng(0).integers(-1000, 1000, 999).astype(np.int64)
    r0 = orc.screen(fv, 0.0)
    assert r0["T"] == r0["mean"]
    assert list(r0["idx"]) == [i for i in range(len(fv)) if fv[i] > fv.sum() / len(fv)]
    assert orc.screen(fv, 1.0)["count"] == 0
    assert orc.screen(np.full(10, 3, np.int64), 0.3)["count"] == 0


# ---------------------------------------------------------------- ascent

def test_ascent_hand_case():
    # Q = [[1,-3],[-3,2]] from x = 00: gains (1, 2) -> flip bit 1 (f = 2);
    # then gains (1 - 6, -2) -> local optimum.  Global optimum is also 2.
    Q = np.array([[1, -3], [-3, 2]], np.int8)
    x, fv, flips, tr = orc.ascent1(Q, np.zeros(1, np.uint64), 0, trace_cap=8)
    assert (int(x[0]), fv, flips, list(tr)) == (0b10, 2, 1, [1])
    assert orc.brute_force(Q)[0] == 2


def test_ascent_tie_goes_to_lowest_index():
    # diagonal 5 everywhere, no coupling: every flip gains 5; order 0,1,2,...
    n = 6
    Q = np.diag(np.full(n, 5, np.int8))
    x, fv, flips, tr = orc.ascent1(Q, np.zeros(1, np.uint64), 0, trace_cap=16)
    assert list(tr) == list(range(n)) and fv == 5 * n and flips == n


@pytest.mark.parametrize("n,density,seed", [(12, 1.0, 1), (40, 0.3, 2), (97, 0.1, 3)])
def test_ascent_steps_are_steepest_flips(n, density, seed):
    Q = synth.make_instance(n, density, seed)
    x = synth.random_solutions(n, 1, seed)[0]
    x01 = synth.unpack_bits(x, n).astype(np.int64)
    f0 = _f_np(Q, x01)
    xn, fn, flips, trace = orc.ascent1(Q, x, f0, trace_cap=10**6)
    assert flips == len(trace)
    cur = x01.copy()
    fc = f0
    for k in trace:
        gains = []
        for i in range(n):
            y = cur.copy()
            y[i] ^= 1
            gains.append(_f_np(Q, y) - fc)
        best = max(gains)
        assert best > 0
        assert k == gains.index(best)  # steepest, lowest index on ties
        cur[k] ^= 1
        fc += best
    # the final point is a local optimum and the running f is exact
    assert fc == fn == _f_np(Q, synth.unpack_bits(xn, n))
    assert np.array_equal(cur, synth.unpack_bits(xn, n))
    for i in range(n):
        y = cur.copy()
        y[i] ^= 1
        assert _f_np(Q, y) <= fc


def test_ascent_max_flips_cap_is_a_prefix():
    n = 60
    Q = synth.make_instance(n, 1.0, 9)
    x = synth.random_solutions(n, 1, 9)[0]
    f0 = _f_np(Q, synth.unpack_bits(x, n))
    _, _, full, tr_full = orc.ascent1(Q, x, f0, trace_cap=10**5)
    assert full > 3
    for cap in (1, 2, 3):
        _, fcap, c, tr = orc.ascent1(Q, x, f0, max_flips=cap, trace_cap=10**5)
        assert c == cap and list(tr) == list(tr_full[:cap])


@pytest.mark.parametrize("n", [8, 14, 18])
def test_ascent_bounded_by_global_optimum(n):
    Q = synth.make_instance(n, 0.6, n)
    gmax, _ = orc.brute_force(Q)
    X = synth.random_solutions(n, 16, n)
    fv = orc.eval(Q, X)
    Xn, fn, flips = orc.ascent(Q, X, fv, np.arange(16, dtype=np.int32))
    assert all(v <= gmax for v in fn)
    assert all(a >= b for a, b in zip(fn, fv))


def test_ascent_only_touches_listed_starts():
    n = 50
    Q = synth.make_instance(n, 0.5, 1)
    X = synth.random_solutions(n, 6, 1)
    fv = orc.eval(Q, X)
    idx = np.array([1, 4], np.int32)
    Xn, fn, flips = orc.ascent(Q, X, fv, idx)
    for s in (0, 2, 3, 5):
        assert np.array_equal(Xn[s], X[s]) and fn[s] == fv[s] and flips[s] == 0
    for s in idx:
        assert fn[s] == _f_np(Q, synth.unpack_bits(Xn[s], n))


# ---------------------------------------------------------------- solve / best

def test_best_lowest_index_on_ties():
    assert orc.best(np.array([3, 9, 1, 9], np.int64)) == (9, 1)


def test_solve_consistency():
    n, S = 100, 200
    Q = synth.make_instance(n, 0.1, 0)
    r = orc.solve(Q, S, 0.5, seed=0)
    assert r["best_f"] == _f_np(Q, synth.unpack_bits(r["best_x"], n))
    assert r["best_f"] >= r["batch_max"]
    x0 = orc.first_derivative(Q)
    X = orc.diversify(x0, n, orc.DIVERSIFY, 0, 0, S)
    fv = orc.eval(Q, X)
    sc = orc.screen(fv, 0.5)
    assert sc["count"] == r["passed"] and sc["max"] == r["batch_max"]
    assert r["passed"] >= 1


@pytest.mark.parametrize("n,S,density,lam,max_flips,seed,mode", [
    (100, 200, 0.1, 0.5, 0, 0, 1),
    (100, 1000, 0.1, 0.5, 0, 0, 1),   # the n = 100 workload in full
    (73, 300, 0.6, 0.25, 0, 7, 1),
    (73, 300, 0.6, 0.75, 3, 7, 1),    # capped climbs
    (130, 257, 1.0, 0.5, 0, 11, 0),   # uniform random starts
])
def test_solve_is_the_round_recomposed_from_its_pinned_steps(n, S, density, lam, max_flips,
                                                             seed, mode):
    # One round of the loop body of Fig. 2 in its order: the first-derivative
    # start, start generation around it, evaluation, the screen, the ascent of
    # the passing starts, then the best over every start's final value.  Each
    # step is pinned on its own above; this pins their composition, so a solve
    # that took the best-of before the ascent, climbed the wrong starts or
    # screened the climbed values fails here.
    Q = synth.make_instance(n, density, seed)
    r = orc.solve(Q, S, lam, max_flips=max_flips, seed=seed, mode=mode)
    x0 = orc.first_derivative(Q)
    X = orc.diversify(x0, n, mode, seed, 0, S)
    fv = orc.eval(Q, X)
    sc = orc.screen(fv, lam)
    Xa, fa, flips = orc.ascent(Q, X, fv, sc["idx"], max_flips)
    bf, bi = orc.best(fa)
    assert r["best_f"] == bf and r["best_index"] == bi
    assert np.array_equal(r["best_x"], Xa[bi])
    assert r["passed"] == sc["count"] and r["batch_max"] == sc["max"]
    assert r["sum"] == int(fv.sum()) and r["T"] == sc["T"] and r["mean"] == sc["mean"]
    assert r["total_flips"] == int(flips.sum())
    assert r["max_flips_seen"] == int(flips.max(initial=0))
    # the climb matters on every case: the best-of taken before the ascent
    # would give a strictly smaller value
    assert bf > int(fv.max())


# ---------------------------------------------------------------- instance generator

def test_instance_generator_shape_and_density():
    n = 400
    for d in (0.1, 1.0):
        Q = synth.make_instance(n, d, 3)
        assert np.array_equal(Q, Q.T)
        assert Q.min() >= -100 and Q.max() <= 100
        nz = np.count_nonzero(np.triu(Q)) / (n * (n + 1) / 2)
        assert abs(nz - d * 200 / 201) < 0.02
    assert orc.validate(synth.make_instance(50, 0.5, 1))[0] == 0
    Q = synth.make_instance(50, 0.5, 1)
    Q[3, 7] += 1
    assert orc.validate(Q)[0] == -2


# ---------------------------------------------------------------- multi-round search

def test_search_pins():
    n = 60
    Q = synth.make_instance(n, 0.4, 2)
    r = orc.search(Q, num_samples=200, S=16, rounds=6, lam=0.5, seed=3)
    # the incumbent only improves, and is the value of the returned solution
    assert all(a <= b for a, b in zip(r["history"], r["history"][1:]))
    assert r["best_f"] == r["history"][-1] == _f_np(Q, synth.unpack_bits(r["best_x"], n))
    # the first start of round 0 is the first-derivative solution, which passes
    # any lambda < 1 screen once the sample mean lies below it, so the result is
    # at least its steepest-ascent local optimum
    x0 = orc.first_derivative(Q)
    f0 = _f_np(Q, synth.unpack_bits(x0, n))
    _, f_loc, _, _ = orc.ascent1(Q, x0, f0)
    assert r["best_f"] >= f_loc
    # the sample mean comes from the random sample: its sum is the oracle's f sum
    Xs = orc.diversify(None, n, orc.RANDOM, 3, 0, 200)
    assert r["sample_sum"] == sum(_f_np(Q, x) for x in synth.unpack_bits(Xs, n))


def test_search_small_n_reaches_a_local_optimum_below_global():
    n = 14
    Q = synth.make_instance(n, 0.8, 5)
    gmax, _ = orc.brute_force(Q)
    r = orc.search(Q, num_samples=64, S=8, rounds=4, lam=0.3, seed=1)
    assert r["best_f"] <= gmax
    x = synth.unpack_bits(r["best_x"], n).astype(np.int64)
    for i in range(n):  # the incumbent is a 1-flip local optimum
        y = x.copy()
        y[i] ^= 1
        assert _f_np(Q, y) <= r["best_f"]


def test_search_replays_the_rounds_of_fig2():
    """The search is the loop of Fig. 2 in rounds: replayed here with numpy
    objective values, a numpy screen and best-of, and the separately pinned
    start generation and ascent."""
    n, S, R, lam, seed, ns = 60, 16, 6, 0.5, 3, 200
    Q = synth.make_instance(n, 0.4, 2)
    r = orc.search(Q, num_samples=ns, S=S, rounds=R, lam=lam, seed=seed)
    sample = synth.unpack_bits(orc.diversify(None, n, orc.RANDOM, seed, 0, ns), n)
    mean = np.float64(sum(_f_np(Q, x) for x in sample)) / np.float64(ns)
    inc = orc.first_derivative(Q)
    inc_f = _f_np(Q, synth.unpack_bits(inc, n))
    history, passed = [], 0
    for rnd in range(R):
        X = orc.diversify(inc, n, orc.DIVERSIFY, seed, rnd, S)
        fv = [_f_np(Q, x) for x in synth.unpack_bits(X, n)]
        T = mean + np.float64(lam) * (np.float64(inc_f) - mean)
        for s in range(S):
            if np.float64(fv[s]) > T:
                X[s], fv[s], _, _ = orc.ascent1(Q, X[s], fv[s])
                passed += 1
        b = int(np.argmax(fv))  # first maximum: lowest index on ties
        if fv[b] > inc_f:
            inc, inc_f = X[b].copy(), fv[b]
        history.append(inc_f)
    assert list(r["history"]) == history
    assert r["best_f"] == inc_f and np.array_equal(r["best_x"], inc)
    assert r["passed"] == passed


# ------------------------------------------------------------ path relinking

def _relink_np(Q, x, g):
    """Path relinking replayed with brute-force gains f(x ^ e_j) - f(x)."""
    x = np.array(x, dtype=np.int64)
    g = np.asarray(g, dtype=np.int64)
    fx = _f_np(Q, x)
    D = int((x != g).sum())
    best_x, best_f, have = x.copy(), fx, False
    for t in range(1, D + 1):
        gains = []
        for j in np.flatnonzero(x != g):
            y = x.copy()
            y[j] ^= 1
            gains.append((_f_np(Q, y) - fx, -j))
        gain, negj = max(gains)  # largest gain, then lowest index
        x[-negj] ^= 1
        fx += gain
        if t < D and (not have or fx > best_f):
            best_x, best_f, have = x.copy(), fx, True
    assert np.array_equal(x, g)  # the path ends at the guiding solution
    return best_x, best_f, D


def test_relink_hand_case():
    # Q = [[1,-2,0],[-2,3,1],[0,1,-1]], from 000 toward 111: gains (1, 3, -1)
    # -> flip 1 (f=3); then y = column 1 = (-2, 3, 1): gains x0: 1 - 4 = -3,
    # x2: -1 + 2 = 1 -> flip 2 (f=4); then x0 (gain -3, f=1 = sum of Q).
    # Intermediates 010 (3) and 011 (4): best 011, value 4, distance 3.
    Q = np.array([[1, -2, 0], [-2, 3, 1], [0, 1, -1]], dtype=np.int8)
    xb, fb, d = orc.relink1(Q, np.array([0], np.uint64), np.array([7], np.uint64))
    assert (int(xb[0]), fb, d) == (0b110, 4, 3)


@pytest.mark.parametrize("n,density,seed", [(9, 1.0, 1), (23, 0.5, 2), (64, 0.3, 3),
                                            (70, 1.0, 4)])
def test_relink_matches_bruteforce_replay(n, density, seed):
    Q = synth.make_instance(n, density, seed)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        x = rng.integers(0, 2, n)
        g = rng.integers(0, 2, n)
        xb, fb, d = orc.relink1(Q, synth.pack_bits(x), synth.pack_bits(g))
        ex, ef, ed = _relink_np(Q, x, g)
        assert d == ed and fb == ef
        assert np.array_equal(synth.unpack_bits(xb, n), ex)
        assert fb == _f_np(Q, synth.unpack_bits(xb, n))


def test_relink_short_distances_return_the_initiating_solution():
    n = 40
    Q = synth.make_instance(n, 0.5, 9)
    x = np.random.default_rng(1).integers(0, 2, n)
    for flip in ([], [17]):
        g = x.copy()
        g[flip] ^= 1
        xb, fb, d = orc.relink1(Q, synth.pack_bits(x), synth.pack_bits(g))
        assert d == len(flip)
        assert np.array_equal(synth.unpack_bits(xb, n), x) and fb == _f_np(Q, x)


def test_relink_batch_is_pairwise():
    n = 50
    Q = synth.make_instance(n, 0.6, 11)
    X = orc.diversify(None, n, orc.RANDOM, 1, 0, 5)
    G = orc.diversify(None, n, orc.RANDOM, 2, 0, 5)
    Xb, fb, d = orc.relink(Q, X, G)
    for p in range(5):
        xb1, fb1, d1 = orc.relink1(Q, X[p], G[p])
        assert np.array_equal(Xb[p], xb1) and fb[p] == fb1 and d[p] == d1
