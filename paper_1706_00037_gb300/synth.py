"""Seeded synthetic inputs: UBQP instances and arbitrary bit-packed solutions.

This module is the only code shared by the callers of the CUDA library and of
the CPU oracle.  It holds none of the method's arithmetic -- no objective, no
screen, no ascent, no start generation -- only the instances the method is run
on and the bit-packing of the solution layout.

Instance recipe (stands in for the ORLIB and Palubeckis instance files, which
are not available): for every pair i <= j draw u = rng(seed, 1, i*n + j); the
pair is nonzero iff (u >> 11) * 2**-53 < density; its value is
((rng(seed, 2, i*n + j) >> 32) * 201 >> 32) - 100, uniform over the 201
integers in [-100, 100]; Q_ij = Q_ji = value.  The diagonal follows the same
rule (linear and quadratic terms share the density, as in the ORLIB set).
rng(seed, stream, ctr) = splitmix64(seed ^ stream * 0x9E3779B97F4A7C15 ^ ctr),
SplitMix64 being the generator of Steele, Lea & Flood (2014).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = 0x9E3779B97F4A7C15


def _mix(state: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = state + np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def rng_array(seed: int, stream: int, ctr: np.ndarray) -> np.ndarray:
    """Vectorised rng(seed, stream, ctr) over a uint64 counter array."""
    key = np.uint64((seed ^ ((stream * GOLDEN) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF)
    return _mix(np.asarray(ctr, dtype=np.uint64) ^ key)


def make_instance(n: int, density: float, seed: int, ldq: int | None = None,
                  rows_per_block: int = 512) -> np.ndarray:
    """Symmetric int8 Q (n x ldq, zero beyond column n) per the recipe above."""
    ldq = n if ldq is None else ldq
    assert ldq >= n
    Q = np.zeros((n, ldq), dtype=np.int8)
    thr = float(density)
    cols = np.arange(n, dtype=np.uint64)
    for r0 in range(0, n, rows_per_block):
        r1 = min(n, r0 + rows_per_block)
        rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
        ctr = rows * np.uint64(n) + cols[None, :]
        u = rng_array(seed, 1, ctr)
        keep = (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) < thr
        v = rng_array(seed, 2, ctr) >> np.uint64(32)
        val = ((v * np.uint64(201)) >> np.uint64(32)).astype(np.int64) - 100
        val = np.where(keep, val, 0).astype(np.int8)
        # keep only i <= j from the drawn block; the mirror comes from below
        upper = rows <= cols[None, :]
        Q[r0:r1, :n] = np.where(upper, val, 0)
    up = Q[:, :n].copy()
    low = np.tril(up.T, -1)
    Q[:, :n] = up + low
    return Q


def words(n: int) -> int:
    return (n + 63) // 64


def pack_bits(x01: np.ndarray) -> np.ndarray:
    """(..., n) array of 0/1 -> (..., ceil(n/64)) uint64, bit j in word j//64."""
    x01 = np.asarray(x01, dtype=np.uint8)
    n = x01.shape[-1]
    W = words(n)
    pad = np.zeros(x01.shape[:-1] + (W * 64,), np.uint8)
    pad[..., :n] = x01
    b = np.packbits(pad.reshape(x01.shape[:-1] + (W, 8, 8)), axis=-1, bitorder="little")
    return np.ascontiguousarray(b.reshape(x01.shape[:-1] + (W, 8))).view(np.uint64).reshape(
        x01.shape[:-1] + (W,))


def unpack_bits(X: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_bits: (..., W) uint64 -> (..., n) uint8 of 0/1."""
    X = np.ascontiguousarray(X, dtype=np.uint64)
    b = X.view(np.uint8).reshape(X.shape[:-1] + (X.shape[-1] * 8,))
    bits = np.unpackbits(b, axis=-1, bitorder="little")
    return bits[..., :n]


def random_solutions(n: int, S: int, seed: int, p_one: float = 0.5) -> np.ndarray:
    """S arbitrary bit-packed solutions (test inputs; bits >= n are zero)."""
    r = np.random.default_rng(seed)
    return pack_bits((r.random((S, n)) < p_one).astype(np.uint8))


# ---------------------------------------------------------------- workloads
# The seeded instance sets of the multi-instance and serving workloads, shared
# by the benchmark and the tests so that both run the same inputs.

def batch_specs(count: int = 64, seed: int = 4) -> list[tuple[int, float, int]]:
    """(n, density, instance seed) of the multi-instance batch: n uniform on
    [200, 2500], density drawn from {0.1, 0.5, 1.0}, instance seeds 1000*seed + k."""
    r = np.random.default_rng(seed)
    ns = r.integers(200, 2501, count)
    ds = r.choice([0.1, 0.5, 1.0], count)
    return [(int(n), float(d), 1000 * seed + k) for k, (n, d) in enumerate(zip(ns, ds))]


SERVE_MASTER_N = 8192


def serve_master(density: float, seed: int = 5) -> np.ndarray:
    """The master instance request instances are cut from (n = 8192)."""
    return make_instance(SERVE_MASTER_N, density, 5000 + seed + (0 if density < 0.5 else 1))


def serve_requests(count: int, seed: int = 5) -> list[tuple[int, float, int]]:
    """(n, density, offset) of `count` requests: n log-uniform on [500, 7000],
    density in {0.1, 1.0}, and the request's instance the principal submatrix
    M[o:o+n, o:o+n] of the master M of that density at an offset o uniform on
    [0, 8192 - n] -- a symmetric instance of the same recipe for every
    request, drawn without building one matrix per request."""
    r = np.random.default_rng(seed)
    ns = np.exp(r.uniform(np.log(500), np.log(7000), count)).astype(int)
    ds = r.choice([0.1, 1.0], count)
    offs = [int(r.integers(0, SERVE_MASTER_N - int(n) + 1)) for n in ns]
    return [(int(n), float(d), o) for n, d, o in zip(ns, ds, offs)]
