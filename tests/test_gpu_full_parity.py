"""Every-element parity with the oracle at the workloads' full sizes.

The oracle runs on every host core (``oracle_pool``), which makes full batches
affordable: every objective value, the whole screen (T, Mean, the sums and the
complete pass set), every climbed start's final solution, value, flip count and
complete sequence of flipped indices (``ubqp_ascent_trace``), and every
instance's or request's result are compared element by element, on the same
seeded inputs, with the CUDA path run in the configuration the benchmark times.

Workloads (see ``paper_1706_00037_gb300.synth``): the Table 1 sizes n = 2500,
5000, 6000, 7000 (dense, 1000 random starts); the benchmark's round at
n = 7000 and the same batch with every start climbed; n = 5000 at density 0.1
with 8192 diversified starts and lambda in {0.25, 0.5, 0.75}; the 64-instance
batch plan; requests of the serving mix.
"""
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


def host_words(t):
    return t.cpu().numpy().view(np.uint64)


def gpu_round(inst, S, lam, mode, seed, ldt, idx_all=False):
    """One round as the benchmark runs it (diversify, eval, screen, ascent with
    the tensor-core start-up and the start counter, best), the ascent traced.
    The untraced ascent of the same starts is run on a copy and must agree."""
    X = ubqp.diversify(inst, S, mode=mode, seed=seed)
    f = ubqp.eval(inst, X)
    X0, f0 = X.clone(), f.clone()
    sc = ubqp.screen(f, lam)
    idx, cnt = sc["idx"], sc["count"]
    if idx_all:
        idx = torch.arange(S, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), S, dtype=torch.int64, device="cuda")
    Xu, fu = X.clone(), f.clone()
    flips_u = torch.zeros(S, dtype=torch.int32, device="cuda")
    ubqp.ascent(inst, Xu, fu, idx, cnt, 0, flips_u)
    flips, trace = ubqp.ascent_trace(inst, X, f, idx, cnt, ldt)
    bx, bf = ubqp.best(f, X)
    inst.sync()
    assert torch.equal(Xu, X) and torch.equal(fu, f) and torch.equal(flips_u, flips)
    c = int(cnt.item())
    return dict(X0=host_words(X0), f0=f0.cpu().numpy(), X=host_words(X), f=f.cpu().numpy(),
                idx=idx[:c].cpu().numpy(), T=float(sc["Tm"][0].item()),
                mean=float(sc["Tm"][1].item()), stats=sc["stats"].cpu().numpy(),
                flips=flips.cpu().numpy(), trace=trace.cpu().numpy().view(np.uint16),
                bx=host_words(bx), bf=bf.cpu().numpy())


def check_screen(r, f_want, lam):
    sc = orc.screen(f_want, lam)
    assert r["T"] == sc["T"] and r["mean"] == sc["mean"]
    assert list(r["stats"]) == [sc["sum"], sc["max"], sc["argmax"]]
    assert np.array_equal(r["idx"], sc["idx"])
    return sc


def check_climbs(r, Xh, f_want, climbed, ldt):
    """Every climbed start against orc.ascent1: solution, value, flip count and
    the whole move sequence; every other start untouched; the best-of."""
    for s, (xw, fw, cw, tw) in climbed.items():
        assert int(r["f"][s]) == fw, s
        assert int(r["flips"][s]) == cw, s
        assert np.array_equal(r["X"][s], xw), s
        k = min(cw, ldt)
        assert np.array_equal(r["trace"][s, :k].astype(np.int64), tw[:k].astype(np.int64)), s
    rest = np.setdiff1d(np.arange(Xh.shape[0]), np.fromiter(climbed.keys(), np.int64))
    assert np.array_equal(r["f"][rest], f_want[rest]) and np.array_equal(r["X"][rest], Xh[rest])
    assert np.all(r["flips"][rest] == 0)
    fa = f_want.copy()
    for s, (_, fw, _, _) in climbed.items():
        fa[s] = fw
    bf, bi = orc.best(fa)
    assert int(r["bf"][0]) == bf and int(r["bf"][1]) == bi
    xb = climbed[bi][0] if bi in climbed else Xh[bi]
    assert np.array_equal(r["bx"], xb)


@pytest.mark.parametrize("n", [2500, 5000, 6000, 7000])
def test_table1_sizes_every_value_every_path(pool, n):
    S = 1000
    Q = synth.make_instance(n, 1.0, n)
    ref = pool.put(Q)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=n + 1)
    Xh = orc.diversify(None, n, orc.RANDOM, n + 1, 0, S)
    assert np.array_equal(host_words(X), Xh)
    want = pool.eval(ref, Xh)
    for path in (ubqp.EVAL_AUTO, ubqp.EVAL_TC, ubqp.EVAL_TC_STAGED, ubqp.EVAL_TC_TMEM,
                 ubqp.EVAL_PLAIN):
        got = ubqp.eval(inst, X, path=path).cpu().numpy()
        assert np.array_equal(got, want), (path, int(np.sum(got != want)))
    inst.sync()


def test_benchmark_round_n7000_every_element(pool):
    # the benchmark's step: n = 7000 dense, 1000 random starts, lambda = 0.5
    n, S, lam = 7000, 1000, 0.5
    seed, ldt = 1_000_003 + 3, 2 * n
    Q = synth.make_instance(n, 1.0, n)
    ref = pool.put(Q)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    r = gpu_round(inst, S, lam, ubqp.RANDOM, seed, ldt)
    Xh = orc.diversify(None, n, orc.RANDOM, seed, 0, S)
    assert np.array_equal(r["X0"], Xh)
    f_want = pool.eval(ref, Xh)
    assert np.array_equal(r["f0"], f_want)
    sc = check_screen(r, f_want, lam)
    assert sc["count"] > 0
    climbed = pool.ascents(ref, Xh, f_want, sc["idx"], cap=ldt)
    assert max(c for _, _, c, _ in climbed.values()) <= ldt
    check_climbs(r, Xh, f_want, climbed, ldt)


def test_every_start_climbed_n7000(pool):
    # the 1-flip moves/s workload: the same instance, 1000 random starts, every
    # start climbed (no screen)
    n, S, ldt = 7000, 1000, 2 * 7000
    Q = synth.make_instance(n, 1.0, n)
    ref = pool.put(Q)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    r = gpu_round(inst, S, 0.5, ubqp.RANDOM, 778, ldt, idx_all=True)
    Xh = orc.diversify(None, n, orc.RANDOM, 778, 0, S)
    f_want = pool.eval(ref, Xh)
    assert np.array_equal(r["f0"], f_want)
    climbed = pool.ascents(ref, Xh, f_want, range(S), cap=ldt)
    check_climbs(r, Xh, f_want, climbed, ldt)
    assert int(r["flips"].sum()) == sum(c for _, _, c, _ in climbed.values())


_SPARSE = {}


def _sparse_case(pool):
    """n = 5000, density 0.1, 8192 starts diversified around the first-derivative
    start: instance, starts and the oracle's values (shared by the three lambdas)."""
    if not _SPARSE:
        n, S = 5000, 8192
        Q = synth.make_instance(n, 0.1, 3)
        ref = pool.put(Q)
        Xh = orc.diversify(orc.first_derivative(Q), n, orc.DIVERSIFY, 3, 0, S)
        _SPARSE.update(Q=Q, ref=ref, Xh=Xh, f=pool.eval(ref, Xh), climbed={})
    return _SPARSE


@pytest.mark.parametrize("lam", [0.25, 0.5, 0.75])
def test_one_large_sparse_instance_every_passer(pool, lam):
    c = _sparse_case(pool)
    n, S, ldt = 5000, 8192, 2 * 5000
    inst = ubqp.Instance(torch.from_numpy(c["Q"]).cuda())
    r = gpu_round(inst, S, lam, ubqp.DIVERSIFY, 3, ldt)
    assert np.array_equal(r["X0"], c["Xh"])
    assert np.array_equal(r["f0"], c["f"])
    sc = check_screen(r, c["f"], lam)
    assert sc["count"] > 0
    # a start's climb does not depend on lambda: climb the new passers only
    todo = [s for s in sc["idx"] if int(s) not in c["climbed"]]
    c["climbed"].update(pool.ascents(c["ref"], c["Xh"], c["f"], todo, cap=ldt))
    climbed = {int(s): c["climbed"][int(s)] for s in sc["idx"]}
    check_climbs(r, c["Xh"], c["f"], climbed, ldt)


def test_batch_plan_every_instance_equals_oracle(pool):
    # 64 instances, n ~ U[200, 2500], density in {0.1, 0.5, 1.0}, 1024 starts
    # each, lambda 0.5: tuned, captured and replayed as the benchmark runs it
    specs = synth.batch_specs()
    Qs = [synth.make_instance(n, d, s) for n, d, s in specs]
    insts = [ubqp.Instance(torch.from_numpy(Q).cuda()) for Q in Qs]
    S, lam, seed = 1024, 0.5, 101
    b = ubqp.Batch(insts, ubqp.make_params(S, lam, seed=0))
    b.tune()
    b.capture()
    b.run(seed)
    torch.cuda.synchronize()
    refs = [pool.put(Q) for Q in Qs]
    want = pool.solves([(ref, S, lam, seed, orc.DIVERSIFY, 0) for ref in refs])
    for i, w in enumerate(want):
        bx, bf = b.result(i)
        assert int(bf[0]) == w["best_f"] and int(bf[1]) == w["best_index"], i
        assert np.array_equal(bx.cpu().numpy().view(np.uint64), w["best_x"]), i
    b.close()


def test_served_requests_equal_oracle(pool):
    # requests of the serving mix (n log-uniform on [500, 7000], density in
    # {0.1, 1.0}, each its own instance), submitted together so that they run
    # concurrently; each result against the oracle's one-round solve
    reqs = synth.serve_requests(24, seed=11)
    masters = {d: synth.serve_master(d) for d in (0.1, 1.0)}
    pinned = {d: torch.from_numpy(M).pin_memory() for d, M in masters.items()}
    S, lam = 1024, 0.5
    srv = ubqp.Server(8, 7000, ubqp.make_params(S, lam, seed=0))
    tickets = []
    for k, (n, d, o) in enumerate(reqs):
        tickets.append(srv.submit(pinned[d], 500 + k, n=n, offset=o))
    res = [srv.wait(t) for t in tickets]
    srv.close()
    for k, (n, d, o) in enumerate(reqs):
        Q = np.ascontiguousarray(masters[d][o:o + n, o:o + n])
        w = pool.solve_recomposed(pool.put(Q), Q, S, lam, 500 + k, orc.DIVERSIFY)
        bf, bx, _ = res[k]
        assert bf == [w["best_f"], w["best_index"]], k
        assert np.array_equal(np.asarray(bx, np.uint64), w["best_x"]), k
