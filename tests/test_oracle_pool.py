"""The multi-process oracle the full-size parity tests use (CPU only): its
pieces equal the oracle's single-process calls, and a round recomposed from
them equals the oracle's own one-round solve."""
import numpy as np

import oracle as orc
from oracle_pool import OraclePool
from paper_1706_00037_gb300 import synth


def test_pool_pieces_and_recomposed_round_equal_the_oracle():
    p = OraclePool(procs=3)
    try:
        n, S, lam, seed = 90, 300, 0.5, 4
        Q = synth.make_instance(n, 0.3, 8)
        ref = p.put(Q)
        X = orc.diversify(orc.first_derivative(Q), n, orc.DIVERSIFY, seed, 0, S)
        f = p.eval(ref, X, chunk=7)
        assert np.array_equal(f, orc.eval(Q, X))
        idx = orc.screen(f, lam)["idx"]
        got = p.ascents(ref, X, f, idx, cap=4 * n)
        for s in idx:
            xw, fw, cw, tw = orc.ascent1(Q, X[s], int(f[s]), 0, 4 * n)
            xg, fg, cg, tg = got[int(s)]
            assert fg == fw and cg == cw and np.array_equal(xg, xw) and np.array_equal(tg, tw)
        for mode in (orc.DIVERSIFY, orc.RANDOM):
            r = p.solve_recomposed(ref, Q, S, lam, seed, mode)
            w = orc.solve(Q, S, lam, seed=seed, mode=mode)
            assert r["best_f"] == w["best_f"] and r["best_index"] == w["best_index"]
            assert np.array_equal(r["best_x"], w["best_x"]) and r["passed"] == w["passed"]
        [w2] = p.solves([(ref, S, lam, seed, orc.DIVERSIFY, 0)])
        assert w2["best_f"] == orc.solve(Q, S, lam, seed=seed)["best_f"]
    finally:
        p.close()
