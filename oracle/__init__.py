"""TEST INFRASTRUCTURE: the CPU oracle of the UBQP hot path.

A thin ctypes wrapper over ``ubqp_oracle.c`` (plain single-threaded C, int64
arithmetic, one FP64 threshold).  The oracle restates the method of Lewis,
arXiv 1706.00037 -- problem (P) of the Introduction and the Pseudocode section
(Fig. 2) -- and is the yardstick every CUDA result is compared against.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The CUDA
library (``paper_1706_00037_gb300``) never does, and the two share no code:
the only module both sides' callers use is the seeded input generator
``paper_1706_00037_gb300.synth``, which holds none of the method's arithmetic.

Every function takes host numpy arrays in the layouts of the C header:
``Q`` is a 2-D int8 array (n rows, row stride = its second dimension >= n),
solutions are bit-packed uint64 words, ``W = ceil(n/64)`` words each, bit ``j``
in word ``j // 64`` at position ``j % 64``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ubqp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libubqp_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(os.path.join(_HERE, f)) > os.path.getmtime(_LIB_PATH)
        for f in ("ubqp_oracle.c", "ubqp_oracle.h"))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "orc_splitmix64": (u64, [u64]),
        "orc_rng": (u64, [u64, u64, u64]),
        "orc_validate": (ctypes.c_int, [P, i32, i64, P]),
        "orc_f": (i64, [P, i32, i64, P]),
        "orc_eval": (None, [P, i32, i64, P, i64, P]),
        "orc_first_derivative": (None, [P, i32, i64, P]),
        "orc_diversify": (None, [P, i32, i32, u64, u64, i64, i32, P]),
        "orc_screen": (None, [P, i64, f64, P, P, P, P, P, P, P]),
        "orc_screen_exact": (ctypes.c_int, [P, i64, f64, P]),
        "orc_ascent1": (i32, [P, i32, i64, P, P, i32, P, i32]),
        "orc_ascent": (None, [P, i32, i64, P, P, P, i64, i32, P]),
        "orc_best": (i64, [P, i64, P]),
        "orc_solve": (None, [P, i32, i64, i64, f64, i32, u64, i32, i32, P, P, P, P]),
        "orc_brute_force": (i64, [P, i32, i64, P]),
        "orc_search": (None, [P, i32, i64, i64, i64, i32, f64, i32, u64, i32, P, P, P, P]),
        "orc_relink1": (i32, [P, i32, i64, P, P, P, P]),
        "orc_relink": (None, [P, i32, i64, P, P, i64, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _q(Q: np.ndarray):
    Q = np.ascontiguousarray(Q, dtype=np.int8)
    assert Q.ndim == 2 and Q.shape[1] >= Q.shape[0]
    return Q, Q.shape[0], Q.shape[1]


def words(n: int) -> int:
    return (n + 63) // 64


RANDOM = 0
DIVERSIFY = 1


def splitmix64(state: int) -> int:
    return int(_load().orc_splitmix64(state & (2**64 - 1)))


def rng(seed: int, stream: int, ctr: int) -> int:
    m = 2**64 - 1
    return int(_load().orc_rng(seed & m, stream & m, ctr & m))


def validate(Q):
    """(status, max|Q|): status 0 = symmetric, -2 = not symmetric."""
    Q, n, ldq = _q(Q)
    m = np.zeros(1, np.int32)
    st = _load().orc_validate(_p(Q), n, ldq, _p(m))
    return int(st), int(m[0])


def f(Q, x) -> int:
    Q, n, ldq = _q(Q)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    return int(_load().orc_f(_p(Q), n, ldq, _p(x)))


def eval(Q, X) -> np.ndarray:  # noqa: A001 - the paper's routine name
    Q, n, ldq = _q(Q)
    X = np.ascontiguousarray(X, dtype=np.uint64).reshape(-1, words(n))
    out = np.zeros(X.shape[0], np.int64)
    _load().orc_eval(_p(Q), n, ldq, _p(X), X.shape[0], _p(out))
    return out


def first_derivative(Q) -> np.ndarray:
    Q, n, ldq = _q(Q)
    x0 = np.zeros(words(n), np.uint64)
    _load().orc_first_derivative(_p(Q), n, ldq, _p(x0))
    return x0


def diversify(x0, n: int, mode: int, seed: int, round_: int, S: int,
              div_H: int = 64) -> np.ndarray:
    W = words(n)
    x0 = np.ascontiguousarray(x0 if x0 is not None else np.zeros(W), dtype=np.uint64)
    X = np.zeros((S, W), np.uint64)
    _load().orc_diversify(_p(x0), n, mode, seed & (2**64 - 1), round_, S, div_H, _p(X))
    return X


def screen(fv, lam: float) -> dict:
    fv = np.ascontiguousarray(fv, dtype=np.int64)
    S = fv.shape[0]
    idx = np.zeros(max(S, 1), np.int32)
    c = np.zeros(1, np.int64)
    T = np.zeros(1, np.float64)
    mean = np.zeros(1, np.float64)
    mx = np.zeros(1, np.int64)
    am = np.zeros(1, np.int64)
    sm = np.zeros(1, np.int64)
    _load().orc_screen(_p(fv), S, float(lam), _p(idx), _p(c), _p(T), _p(mean),
                       _p(mx), _p(am), _p(sm))
    k = int(c[0])
    return {"idx": idx[:k].copy(), "count": k, "T": float(T[0]),
            "mean": float(mean[0]), "max": int(mx[0]), "argmax": int(am[0]),
            "sum": int(sm[0])}


def screen_exact(fv, lam: float) -> np.ndarray:
    fv = np.ascontiguousarray(fv, dtype=np.int64)
    out = np.zeros(fv.shape[0], np.uint8)
    st = _load().orc_screen_exact(_p(fv), fv.shape[0], float(lam), _p(out))
    if st != 0:
        raise ValueError("lambda outside the exact check's range")
    return out.astype(bool)


def ascent1(Q, x, fx: int, max_flips: int = 0, trace_cap: int = 0):
    """Returns (x_new, f_new, flips, trace)."""
    Q, n, ldq = _q(Q)
    x = np.array(x, dtype=np.uint64, copy=True)
    fv = np.array([fx], np.int64)
    tr = np.zeros(max(trace_cap, 1), np.int32)
    c = _load().orc_ascent1(_p(Q), n, ldq, _p(x), _p(fv), max_flips, _p(tr), trace_cap)
    return x, int(fv[0]), int(c), tr[:min(c, trace_cap)].copy()


def ascent(Q, X, fv, idx, max_flips: int = 0):
    """Returns (X_new, f_new, flips) with flips zero for starts not in idx."""
    Q, n, ldq = _q(Q)
    X = np.array(X, dtype=np.uint64, copy=True).reshape(-1, words(n))
    fv = np.array(fv, dtype=np.int64, copy=True)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    flips = np.zeros(X.shape[0], np.int32)
    _load().orc_ascent(_p(Q), n, ldq, _p(X), _p(fv), _p(idx), idx.shape[0],
                       max_flips, _p(flips))
    return X, fv, flips


def best(fv):
    fv = np.ascontiguousarray(fv, dtype=np.int64)
    bi = np.zeros(1, np.int64)
    v = _load().orc_best(_p(fv), fv.shape[0], _p(bi))
    return int(v), int(bi[0])


def solve(Q, S: int, lam: float, max_flips: int = 0, seed: int = 0,
          mode: int = DIVERSIFY, div_H: int = 64) -> dict:
    Q, n, ldq = _q(Q)
    bx = np.zeros(words(n), np.uint64)
    bf = np.zeros(1, np.int64)
    st = np.zeros(6, np.int64)
    sf = np.zeros(2, np.float64)
    _load().orc_solve(_p(Q), n, ldq, S, float(lam), max_flips, seed & (2**64 - 1),
                      mode, div_H, _p(bx), _p(bf), _p(st), _p(sf))
    return {"best_x": bx, "best_f": int(bf[0]), "passed": int(st[0]),
            "total_flips": int(st[1]), "max_flips_seen": int(st[2]),
            "batch_max": int(st[3]), "best_index": int(st[4]), "sum": int(st[5]),
            "T": float(sf[0]), "mean": float(sf[1])}


def search(Q, num_samples: int, S: int, rounds: int, lam: float, max_flips: int = 0,
           seed: int = 0, div_H: int = 64) -> dict:
    """Multi-round search of Fig. 2 (see ubqp_oracle.c)."""
    Q, n, ldq = _q(Q)
    bx = np.zeros(words(n), np.uint64)
    bf = np.zeros(1, np.int64)
    hist = np.zeros(max(rounds, 1), np.int64)
    st = np.zeros(3, np.int64)
    _load().orc_search(_p(Q), n, ldq, num_samples, S, rounds, float(lam), max_flips,
                       seed & (2**64 - 1), div_H, _p(bx), _p(bf), _p(hist), _p(st))
    return {"best_x": bx, "best_f": int(bf[0]), "history": hist[:rounds].copy(),
            "passed": int(st[0]), "total_flips": int(st[1]), "sample_sum": int(st[2])}


def relink1(Q, x, g):
    """Path relinking from x toward g: (best intermediate x, its f, distance)."""
    Q, n, ldq = _q(Q)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint64)
    xb = np.zeros(words(n), np.uint64)
    fb = np.zeros(1, np.int64)
    d = _load().orc_relink1(_p(Q), n, ldq, _p(x), _p(g), _p(xb), _p(fb))
    return xb, int(fb[0]), int(d)


def relink(Q, X, G):
    """relink1 over pairs (X[p], G[p]): (X_best, f_best, dist)."""
    Q, n, ldq = _q(Q)
    X = np.ascontiguousarray(X, dtype=np.uint64).reshape(-1, words(n))
    G = np.ascontiguousarray(G, dtype=np.uint64).reshape(-1, words(n))
    P = X.shape[0]
    Xb = np.zeros_like(X)
    fb = np.zeros(P, np.int64)
    d = np.zeros(P, np.int32)
    _load().orc_relink(_p(Q), n, ldq, _p(X), _p(G), P, _p(Xb), _p(fb), _p(d))
    return Xb, fb, d


def brute_force(Q):
    """(global max, lowest maximiser as an int bit pattern); n <= 24."""
    Q, n, ldq = _q(Q)
    assert n <= 24
    b = np.zeros(1, np.uint64)
    v = _load().orc_brute_force(_p(Q), n, ldq, _p(b))
    return int(v), int(b[0])
