"""TEST INFRASTRUCTURE: the CPU oracle spread over every host core.

The oracle (``oracle/``) is plain single-threaded C.  To compare every element
of a full-size batch with it, the tests run it in one spawned process per host
core: instances are placed once in shared memory, and the work is split into
independent pieces that the oracle's own functions compute -- the evaluation of
a chunk of starts, the steepest ascent (with its move record) of one start, a
whole one-round solve of one instance.  A round of Fig. 2 is recomposed from
these pieces in the order of the loop body (first-derivative start, starts,
evaluation, screen, ascent of the passers, best-of); the oracle's pins check
that this recomposition equals its own one-round ``orc_solve``.

Nothing here touches a GPU or the CUDA library; the processes are started
with ``spawn``.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

import oracle as orc

_ATT: dict = {}  # worker side: attached shared instances by name


def _q(ref):
    name, shape = ref
    if name not in _ATT:
        shm = shared_memory.SharedMemory(name=name)
        _ATT[name] = (shm, np.ndarray(shape, dtype=np.int8, buffer=shm.buf))
    return _ATT[name][1]


def _w_eval(args):
    ref, X = args
    return orc.eval(_q(ref), X)


def _w_ascent(args):
    ref, x, fx, max_flips, cap = args
    xn, fn, c, tr = orc.ascent1(_q(ref), x, int(fx), max_flips, cap)
    return xn, fn, c, tr


def _w_solve(args):
    ref, S, lam, seed, mode, max_flips = args
    return orc.solve(_q(ref), S, lam, max_flips=max_flips, seed=seed, mode=mode)


class OraclePool:
    """One spawned process per host core plus instances in shared memory."""

    def __init__(self, procs: int | None = None):
        self.procs = procs or os.cpu_count() or 1
        self._pool = mp.get_context("spawn").Pool(self.procs)
        self._shm: list = []

    def close(self):
        self._pool.terminate()
        self._pool.join()
        for shm in self._shm:
            shm.close()
            shm.unlink()
        self._shm = []

    def put(self, Q: np.ndarray):
        """Share instance Q (copied once); returns the reference the calls take."""
        Q = np.ascontiguousarray(Q, dtype=np.int8)
        shm = shared_memory.SharedMemory(create=True, size=max(Q.nbytes, 1))
        np.ndarray(Q.shape, dtype=np.int8, buffer=shm.buf)[...] = Q
        self._shm.append(shm)
        return (shm.name, Q.shape)

    def eval(self, ref, X: np.ndarray, chunk: int = 16) -> np.ndarray:
        parts = [X[i:i + chunk] for i in range(0, X.shape[0], chunk)]
        out = self._pool.map(_w_eval, [(ref, p) for p in parts], chunksize=1)
        return np.concatenate(out) if out else np.zeros(0, np.int64)

    def ascents(self, ref, X: np.ndarray, f: np.ndarray, idx, max_flips: int = 0,
                cap: int = 0) -> dict:
        """orc.ascent1 of every start X[s], s in idx: {s: (x, f, flips, trace)}."""
        idx = [int(s) for s in idx]
        res = self._pool.map(_w_ascent, [(ref, X[s], int(f[s]), max_flips, cap) for s in idx],
                             chunksize=1)
        return dict(zip(idx, res))

    def solves(self, jobs) -> list:
        """orc.solve for each (ref, S, lam, seed, mode, max_flips), one job per process."""
        return self._pool.map(_w_solve, list(jobs), chunksize=1)

    def solve_recomposed(self, ref, Q: np.ndarray, S: int, lam: float, seed: int,
                         mode: int, max_flips: int = 0) -> dict:
        """One round of the loop body of Fig. 2 from the oracle's pieces, the
        evaluation and the climbs spread over the processes."""
        n = Q.shape[0]
        x0 = orc.first_derivative(Q)
        X = orc.diversify(x0, n, mode, seed, 0, S)
        f = self.eval(ref, X)
        sc = orc.screen(f, lam)
        climbed = self.ascents(ref, X, f, sc["idx"], max_flips)
        Xa, fa = X.copy(), f.copy()
        for s, (x, fv, _, _) in climbed.items():
            Xa[s], fa[s] = x, fv
        bf, bi = orc.best(fa)
        return {"best_f": bf, "best_index": bi, "best_x": Xa[bi], "passed": sc["count"]}
