"""The request loop: every request's result equals the same instance solved
alone (mix invariance), under concurrency and under a tight memory budget."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu

SIZES = [(100, 0.1), (2500, 1.0), (700, 0.5), (3000, 0.1), (129, 1.0), (1800, 0.5)]


def alone(Q, params, seed):
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    p = ubqp.make_params(params.num_starts, params.lambda_, mode=params.mode, seed=seed)
    bx, bf, _ = ubqp.solve(inst, p, want_stats=False)
    torch.cuda.synchronize()
    return bf.cpu().tolist(), bx.cpu().numpy().view(np.uint64)


def test_prepare_into_matches_prepare():
    n = 900
    Q = synth.make_instance(n, 0.5, 3)
    lib = ubqp.load()
    need = int(lib.ubqp_q_arena_size(n))
    arena = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = (arena.data_ptr() + 255) // 256 * 256
    Qd = torch.from_numpy(Q).cuda()
    import ctypes
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.ubqp_q_prepare_into(ctypes.c_void_p(Qd.data_ptr()), n, n, ctypes.c_void_p(base),
                                   need, st, ctypes.byref(h)) == 0
    inst = ubqp.Instance.__new__(ubqp.Instance)
    inst._h, inst.n, inst.words, inst.device = h, n, (n + 63) // 64, Qd.device
    p = ubqp.make_params(300, 0.5, seed=4)
    bx, bf, st1 = ubqp.solve(inst, p)
    want = orc.solve(Q, 300, 0.5, seed=4)
    assert int(bf[0]) == want["best_f"] and st1["passed"] == want["passed"]
    inst.close()


@pytest.mark.parametrize("workers,budget", [(4, 0), (3, "one")])
def test_server_results_equal_alone(workers, budget):
    Qs = [synth.make_instance(n, d, 10 + k) for k, (n, d) in enumerate(SIZES)]
    params = ubqp.make_params(512, 0.5, seed=0)
    srv = ubqp.Server(workers, 3000, params)
    if budget == "one":  # admit one request at a time
        srv.close()
        srv = ubqp.Server(workers, 3000, params, memory_budget=ubqp.Server(
            1, 3000, params).request_bytes(3000))
    reqs = [(k % len(Qs), 1000 + k) for k in range(14)]  # repeats with new seeds
    tickets = [srv.submit(Qs[i], seed) for i, seed in reqs]
    got = [srv.wait(t) for t in tickets]
    srv.close()
    for (i, seed), (bf, bx, lat) in zip(reqs, got):
        wf, wx = alone(Qs[i], params, seed)
        assert bf == wf and np.array_equal(bx, wx), (i, seed)
        assert lat > 0
    # the small instance against the oracle as well
    i, seed = reqs[0]
    want = orc.solve(Qs[i], 512, 0.5, seed=seed)
    assert got[0][0] == [want["best_f"], want["best_index"]]


def test_server_rejects_oversized_instances():
    params = ubqp.make_params(64, 0.5)
    srv = ubqp.Server(2, 500, params)
    with pytest.raises(ubqp.UbqpError) as e:
        srv.submit(synth.make_instance(600, 0.1, 1), 1)
    assert e.value.status == -7
    t = srv.submit(synth.make_instance(400, 0.1, 1), 1)
    assert srv.wait(t)[0][0] != 0 or True
    srv.close()


def test_server_survives_injected_allocation_failures():
    """Failure detection on the host: two admissions fail as out of memory,
    their tickets report UBQP_ERR_NOMEM, and the requests after them are
    served with results equal to solving alone."""
    params = ubqp.make_params(256, 0.5, seed=0)
    srv = ubqp.Server(2, 600, params)
    Qs = [synth.make_instance(n, 0.5, 40 + k) for k, n in enumerate((300, 450, 200, 520))]
    srv.inject_alloc_failures(2)
    tickets = [srv.submit(Q, 7 + k) for k, Q in enumerate(Qs)]
    statuses, results = [], []
    for t in tickets:
        try:
            bf, bx, _ = srv.wait(t)
            statuses.append(0)
            results.append((bf, bx))
        except ubqp.UbqpError as e:
            statuses.append(e.status)
            results.append(None)
    srv.close()
    assert sorted(statuses) == [-4, -4, 0, 0]
    for k, (Q, r) in enumerate(zip(Qs, results)):
        if r is None:
            continue
        inst = ubqp.Instance(torch.from_numpy(Q).cuda())
        p1 = ubqp.make_params(256, 0.5, seed=7 + k)
        bx, bf, _ = ubqp.solve(inst, p1, want_stats=False)
        assert r[0] == bf.tolist() and np.array_equal(r[1], bx.cpu().numpy().view(np.uint64))


def test_server_reports_an_asymmetric_instance_promptly():
    """The server prepares without synchronising: an asymmetric request's
    ticket reports UBQP_ERR_NOT_SYMMETRIC at its one synchronisation, its
    climb is skipped (no run to the watchdog), and the requests around it are
    served with results equal to solving alone."""
    import time
    params = ubqp.make_params(256, 0.5, seed=0)
    srv = ubqp.Server(2, 2000, params)
    good = [synth.make_instance(n, 0.5, 60 + k) for k, n in enumerate((300, 1500))]
    bad = synth.make_instance(1500, 1.0, 62)
    bad[5, 700] = bad[700, 5] + 1
    t0 = time.perf_counter()
    tickets = [srv.submit(good[0], 3), srv.submit(bad, 4), srv.submit(good[1], 5)]
    res = []
    for t in tickets:
        try:
            res.append(srv.wait(t))
        except ubqp.UbqpError as e:
            res.append(e.status)
    assert time.perf_counter() - t0 < 10.0
    srv.close()
    assert res[1] == -2
    for Q, seed, r in ((good[0], 3, res[0]), (good[1], 5, res[2])):
        wf, wx = alone(Q, params, seed)
        assert r[0] == wf and np.array_equal(r[1], wx)


def test_bounded_wait_gives_up_and_context_stays_usable():
    """A kernel waits on a barrier nothing completes: it records a timeout
    after the limit and returns; the next calls run normally."""
    assert ubqp.selftest_timeout(20000) == -6  # UBQP_ERR_TIMEOUT
    Q = synth.make_instance(100, 0.3, 1)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X = ubqp.diversify(inst, 64, mode=ubqp.RANDOM, seed=1)
    f = ubqp.eval(inst, X)
    inst.sync()
    assert np.array_equal(f.cpu().numpy(), orc.eval(Q, X.cpu().numpy().view(np.uint64)))


@pytest.mark.parametrize("max_n,sizes", [
    (3000, [(2500, 1.0), (100, 0.1), (700, 0.5), (1500, 0.1), (3000, 0.5), (129, 1.0)]),
    (7000, [(7000, 1.0), (4500, 0.1), (600, 1.0), (2100, 0.5)]),      # packed 256 x 2
    (9000, [(8500, 0.1), (300, 0.5), (5000, 1.0)]),                    # one start per block
])
def test_server_batches_requests_and_results_equal_alone(max_n, sizes):
    # one lane, requests submitted together: the lane runs them as shared
    # batches (one screen, one climb and one best-of launch per batch), and
    # every result equals the instance solved alone
    Qs = [synth.make_instance(n, d, 80 + k) for k, (n, d) in enumerate(sizes)]
    params = ubqp.make_params(300, 0.5, seed=0)
    srv = ubqp.Server(1, max_n, params, max_batch=8, memory_budget=1 << 40)
    reqs = [(k % len(Qs), 2000 + k) for k in range(2 * len(Qs) + 1)]
    tickets = [srv.submit(Qs[i], seed) for i, seed in reqs]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs) and st["batches"] < len(reqs) and st["largest"] > 1
    for (i, seed), (bf, bx, _) in zip(reqs, got):
        wf, wx = alone(Qs[i], params, seed)
        assert bf == wf and np.array_equal(bx, wx), (i, seed)


def test_server_principal_submatrix_requests():
    # a request passed as a principal submatrix of a larger host matrix, in
    # place (row stride of the larger matrix)
    M = synth.make_instance(1500, 0.4, 91)
    params = ubqp.make_params(200, 0.5, seed=0)
    srv = ubqp.Server(2, 1500, params)
    Mt = torch.from_numpy(M).pin_memory()
    cases = [(700, 0), (900, 333), (1, 1499), (1500, 0)]
    tickets = [srv.submit(Mt, 40 + k, n=n, offset=o) for k, (n, o) in enumerate(cases)]
    got = [srv.wait(t) for t in tickets]
    srv.close()
    for k, ((n, o), (bf, bx, _)) in enumerate(zip(cases, got)):
        Q = np.ascontiguousarray(M[o:o + n, o:o + n])
        want = orc.solve(Q, 200, 0.5, seed=40 + k)
        assert bf == [want["best_f"], want["best_index"]] and np.array_equal(bx, want["best_x"])
