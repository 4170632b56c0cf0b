"""Python binding of libubqp (the C ABI in include/ubqp.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  If the
library cannot be built or loaded this module raises -- there is no fallback.

Solutions are bit-packed uint64 words; torch has no general uint64 support, so
they travel in ``torch.int64`` tensors of shape (S, W) holding the same bits.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

RANDOM, DIVERSIFY = 0, 1
EVAL_AUTO, EVAL_TC, EVAL_PLAIN, EVAL_TC_STAGED, EVAL_TC_TMEM = 0, 1, 2, 3, 4

OK = 0
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_NOT_SYMMETRIC", -3: "ERR_RANGE",
                -4: "ERR_NOMEM", -5: "ERR_CUDA", -6: "ERR_TIMEOUT", -7: "ERR_UNSUPPORTED"}

EXPORTS = ["ubqp_strerror", "ubqp_last_error", "ubqp_abi_version", "ubqp_q_prepare",
           "ubqp_q_destroy", "ubqp_q_info", "ubqp_sync", "ubqp_first_derivative",
           "ubqp_diversify", "ubqp_diversify_range", "ubqp_eval_workspace_size", "ubqp_eval",
           "ubqp_eval_noalloc", "ubqp_screen", "ubqp_screen_stats", "ubqp_screen_apply",
           "ubqp_ascent_workspace_size", "ubqp_ascent", "ubqp_best", "ubqp_solve_workspace_size",
           "ubqp_solve", "ubqp_search_workspace_size", "ubqp_search", "ubqp_batch_create",
           "ubqp_batch_destroy", "ubqp_batch_run", "ubqp_batch_tune", "ubqp_batch_capture",
           "ubqp_batch_result", "ubqp_batch_get", "ubqp_batch_config", "ubqp_q_arena_size",
           "ubqp_q_prepare_into", "ubqp_server_create", "ubqp_server_submit", "ubqp_server_wait",
           "ubqp_server_poll", "ubqp_server_request_bytes", "ubqp_server_destroy",
           "ubqp_relink_workspace_size", "ubqp_relink", "ubqp_server_inject_alloc_failures",
           "ubqp_selftest_timeout", "ubqp_search_resume", "ubqp_q_prepare_into_async",
           "ubqp_ascent_trace", "ubqp_peak_l2_read", "ubqp_peak_int32_ops", "ubqp_peak_int32",
           "ubqp_batch_schedule", "ubqp_batch_set", "ubqp_server_stats",
           "ubqp_solve_rounds_workspace_size", "ubqp_solve_rounds"]


class UbqpError(RuntimeError):
    def __init__(self, status: int, detail: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")


class Params(ctypes.Structure):
    _fields_ = [("num_starts", ctypes.c_int64), ("lambda_", ctypes.c_double),
                ("max_flips", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("round", ctypes.c_uint64),
                ("div_H", ctypes.c_int32), ("eval_path", ctypes.c_int32)]


class SearchParams(ctypes.Structure):
    _fields_ = [("num_samples", ctypes.c_int64), ("starts_per_round", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("max_flips", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("div_H", ctypes.c_int32), ("eval_path", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_n", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("params", Params),
                ("max_batch", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("passed", ctypes.c_int64), ("total_flips", ctypes.c_int64),
                ("max_flips_seen", ctypes.c_int64), ("batch_max", ctypes.c_int64),
                ("best_index", ctypes.c_int64), ("sum", ctypes.c_int64),
                ("T", ctypes.c_double), ("mean", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Build (if stale) and load libubqp.so; raise if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libubqp.so missing at {path}")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sz, f64 = ctypes.c_size_t, ctypes.c_double
    sig = {
        "ubqp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "ubqp_last_error": (ctypes.c_char_p, []),
        "ubqp_abi_version": (ctypes.c_int, []),
        "ubqp_q_prepare": (ctypes.c_int, [P, i32, i64, P, ctypes.POINTER(P)]),
        "ubqp_q_destroy": (None, [P]),
        "ubqp_q_info": (ctypes.c_int, [P, P, P, P, P, P]),
        "ubqp_sync": (ctypes.c_int, [P, P]),
        "ubqp_first_derivative": (ctypes.c_int, [P, P, P]),
        "ubqp_diversify": (ctypes.c_int, [P, P, i32, u64, u64, i64, i32, P, P]),
        "ubqp_diversify_range": (ctypes.c_int, [P, P, i32, u64, u64, i64, i64, i64, i32, P, P]),
        "ubqp_eval_workspace_size": (sz, [P, i64, i32]),
        "ubqp_eval": (ctypes.c_int, [P, P, i64, P, i32, P, sz, P]),
        "ubqp_eval_noalloc": (ctypes.c_int, [P, P, i64, P, P]),
        "ubqp_screen": (ctypes.c_int, [P, i64, f64, P, P, P, P, P]),
        "ubqp_screen_stats": (ctypes.c_int, [P, i64, i64, P, P]),
        "ubqp_screen_apply": (ctypes.c_int, [P, i64, P, i64, f64, P, P, P, P]),
        "ubqp_ascent_workspace_size": (sz, [P, i64]),
        "ubqp_ascent": (ctypes.c_int, [P, P, P, P, P, i64, i32, P, P, sz, P]),
        "ubqp_ascent_trace": (ctypes.c_int, [P, P, P, P, P, i64, i32, P, P, i64, P, sz, P]),
        "ubqp_best": (ctypes.c_int, [P, P, i64, i32, P, P, P]),
        "ubqp_relink_workspace_size": (sz, [P, i64, i32]),
        "ubqp_server_inject_alloc_failures": (ctypes.c_int, [P, i32]),
        "ubqp_selftest_timeout": (ctypes.c_int, [ctypes.c_uint32, P, P]),
        "ubqp_relink": (ctypes.c_int, [P, P, P, P, i64, P, P, P, P, sz, P]),
        "ubqp_solve_workspace_size": (sz, [P, ctypes.POINTER(Params)]),
        "ubqp_solve": (ctypes.c_int, [P, ctypes.POINTER(Params), P, P, ctypes.POINTER(Stats),
                                      P, sz, P]),
        "ubqp_solve_rounds_workspace_size": (sz, [P, ctypes.POINTER(Params), i32]),
        "ubqp_solve_rounds": (ctypes.c_int, [P, ctypes.POINTER(Params), i32, P, P, P, sz, P]),
        "ubqp_search_workspace_size": (sz, [P, ctypes.POINTER(SearchParams)]),
        "ubqp_search": (ctypes.c_int, [P, ctypes.POINTER(SearchParams), P, P, P, P, P, sz, P]),
        "ubqp_search_resume": (ctypes.c_int, [P, ctypes.POINTER(SearchParams), i32, P, P, P, P,
                                              P, sz, P]),
        "ubqp_batch_create": (ctypes.c_int, [P, i32, ctypes.POINTER(Params), ctypes.POINTER(P)]),
        "ubqp_batch_destroy": (None, [P]),
        "ubqp_batch_run": (ctypes.c_int, [P, u64, P]),
        "ubqp_batch_tune": (ctypes.c_int, [P, P]),
        "ubqp_batch_capture": (ctypes.c_int, [P, P]),
        "ubqp_batch_result": (ctypes.c_int, [P, i32, ctypes.POINTER(P), ctypes.POINTER(P)]),
        "ubqp_batch_config": (ctypes.c_int, [P, P, P, P, P, P]),
        "ubqp_batch_schedule": (ctypes.c_int, [P, P, P, P]),
        "ubqp_batch_set": (ctypes.c_int, [P, i32, i32, i32, i32, i32]),
        "ubqp_batch_get": (ctypes.c_int, [P, i32, P, P, P]),
        "ubqp_q_arena_size": (sz, [i32]),
        "ubqp_q_prepare_into": (ctypes.c_int, [P, i32, i64, P, sz, P, ctypes.POINTER(P)]),
        "ubqp_q_prepare_into_async": (ctypes.c_int, [P, i32, i64, P, sz, P, ctypes.POINTER(P)]),
        "ubqp_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]),
        "ubqp_server_submit": (ctypes.c_int, [P, P, i32, i64, u64, ctypes.POINTER(i64)]),
        "ubqp_server_wait": (ctypes.c_int, [P, i64, P, P, ctypes.POINTER(f64)]),
        "ubqp_server_poll": (ctypes.c_int, [P, i64, ctypes.POINTER(i32)]),
        "ubqp_server_request_bytes": (sz, [P, i32]),
        "ubqp_server_destroy": (None, [P]),
        "ubqp_server_stats": (ctypes.c_int, [P, P, P, P]),
        "ubqp_peak_l2_read": (ctypes.c_int, [P, sz, i32, P, P]),
        "ubqp_peak_int32_ops": (i64, [i32, i64]),
        "ubqp_peak_int32": (ctypes.c_int, [i32, i64, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        detail = load().ubqp_last_error().decode()
        raise UbqpError(status, detail or load().ubqp_strerror(status).decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None, pinned_ok: bool = False):
    if t is None:
        return None
    if not (t.is_cuda or (pinned_ok and t.is_pinned())):
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def words(n: int) -> int:
    return (n + 63) // 64


def arena_size(n: int) -> int:
    """Device bytes ubqp_q_prepare_into needs for an instance of size n."""
    return int(load().ubqp_q_arena_size(n))


class Instance:
    """A prepared UBQP instance (device-resident Q); wraps ``ubqp_q*``."""

    def __init__(self, Q: torch.Tensor, stream=None, arena: torch.Tensor | None = None,
                 defer_validation: bool = False):
        """Prepare Q (ubqp_q_prepare); with `arena` (a uint8 CUDA tensor of at
        least arena_size(n) bytes, kept alive by the caller) the prepared copies
        are carved from it instead of new device allocations
        (ubqp_q_prepare_into).  Q may be a CUDA tensor or a pinned CPU tensor,
        which the preparing kernel reads in place.  defer_validation (with an
        arena): ubqp_q_prepare_into_async -- nothing waits for the preparation;
        the symmetry check is reported by the first sync() (max_abs is -1
        until then)."""
        if defer_validation and arena is None:
            raise ValueError("defer_validation needs an arena")
        if Q.dtype != torch.int8 or Q.dim() != 2 or not (Q.is_cuda or Q.is_pinned()):
            raise ValueError("Q must be a 2-D int8 CUDA tensor or pinned CPU tensor")
        Q = Q.contiguous()
        n, ldq = Q.shape
        h = ctypes.c_void_p()
        if arena is None:
            _check(load().ubqp_q_prepare(_ptr(Q, pinned_ok=True), n, ldq, _stream(stream),
                                         ctypes.byref(h)))
        else:
            fn = load().ubqp_q_prepare_into_async if defer_validation else \
                load().ubqp_q_prepare_into
            _check(fn(_ptr(Q, pinned_ok=True), n, ldq, _ptr(arena), arena.numel(),
                      _stream(stream), ctypes.byref(h)))
        self._h = h
        vals = [ctypes.c_int32() for _ in range(4)] + [ctypes.c_int64()]
        _check(load().ubqp_q_info(h, *[ctypes.byref(v) for v in vals]))
        self.n, self.words, self.n_pad, self.max_abs = (v.value for v in vals[:4])
        self.device_bytes = vals[4].value
        self.device = Q.device if Q.is_cuda else torch.device("cuda", torch.cuda.current_device())

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("instance closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().ubqp_q_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """ubqp_sync: wait for `stream`, report kernel errors and a deferred
        validation (then max_abs is known)."""
        _check(load().ubqp_sync(self.handle, _stream(stream)))
        if self.max_abs < 0:
            m = ctypes.c_int32()
            _check(load().ubqp_q_info(self.handle, None, None, None, ctypes.byref(m), None))
            self.max_abs = m.value


def first_derivative(inst: Instance, stream=None) -> torch.Tensor:
    x0 = torch.empty(inst.words, dtype=torch.int64, device=inst.device)
    _check(load().ubqp_first_derivative(inst.handle, _ptr(x0), _stream(stream)))
    return x0


def diversify(inst: Instance, S: int, mode: int = DIVERSIFY, seed: int = 0, round_: int = 0,
              div_H: int = 64, x0: torch.Tensor | None = None, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    X = out if out is not None else torch.empty((S, inst.words), dtype=torch.int64,
                                                device=inst.device)
    _check(load().ubqp_diversify(inst.handle, _ptr(x0), mode, seed % 2**64, round_, S, div_H,
                                 _ptr(X), _stream(stream)))
    return X


def diversify_range(inst: Instance, S_total: int, s_begin: int, S_local: int,
                    mode: int = DIVERSIFY, seed: int = 0, round_: int = 0, div_H: int = 64,
                    x0: torch.Tensor | None = None, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    X = out if out is not None else torch.empty((S_local, inst.words), dtype=torch.int64,
                                                device=inst.device)
    _check(load().ubqp_diversify_range(inst.handle, _ptr(x0), mode, seed % 2**64, round_,
                                       S_total, s_begin, S_local, div_H, _ptr(X),
                                       _stream(stream)))
    return X


def screen_stats(f: torch.Tensor, offset: int = 0, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """{sum, max, lowest argmax + offset} of f (int64[3], on f's device)."""
    st = out if out is not None else torch.empty(3, dtype=torch.int64, device=f.device)
    _check(load().ubqp_screen_stats(_ptr(f), f.shape[0], offset, _ptr(st), _stream(stream)))
    return st


def screen_apply(f: torch.Tensor, gstats: torch.Tensor, S_total: int, lam: float,
                 stream=None) -> dict:
    S = f.shape[0]
    dev = f.device
    idx = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)
    Tm = torch.empty(2, dtype=torch.float64, device=dev)
    _check(load().ubqp_screen_apply(_ptr(f), S, _ptr(gstats), S_total, float(lam), _ptr(idx),
                                    _ptr(count), _ptr(Tm), _stream(stream)))
    return {"idx": idx, "count": count, "Tm": Tm}


def eval_workspace_size(inst: Instance, S: int, path: int = EVAL_AUTO) -> int:
    return int(load().ubqp_eval_workspace_size(inst.handle, S, path))


def eval(inst: Instance, X: torch.Tensor, path: int = EVAL_AUTO, out: torch.Tensor | None = None,
         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:  # noqa: A001
    S = X.shape[0]
    f = out if out is not None else torch.empty(S, dtype=torch.int64, device=inst.device)
    need = eval_workspace_size(inst, S, path)
    if ws is None and need:
        ws = torch.empty(need, dtype=torch.uint8, device=inst.device)
    nbytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(load().ubqp_eval(inst.handle, _ptr(X), S, _ptr(f), path, _ptr(ws), nbytes,
                            _stream(stream)))
    return f


def eval_noalloc(inst: Instance, X: torch.Tensor, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """Tensor-core evaluation with the library's built-in static scratch
    (no workspace, no device allocation inside the library)."""
    S = X.shape[0]
    f = out if out is not None else torch.empty(S, dtype=torch.int64, device=inst.device)
    _check(load().ubqp_eval_noalloc(inst.handle, _ptr(X), S, _ptr(f), _stream(stream)))
    return f


def screen(f: torch.Tensor, lam: float, stream=None) -> dict:
    S = f.shape[0]
    dev = f.device
    idx = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)
    Tm = torch.empty(2, dtype=torch.float64, device=dev)
    st = torch.empty(3, dtype=torch.int64, device=dev)
    _check(load().ubqp_screen(_ptr(f), S, float(lam), _ptr(idx), _ptr(count), _ptr(Tm),
                              _ptr(st), _stream(stream)))
    return {"idx": idx, "count": count, "Tm": Tm, "stats": st}


def ascent_workspace_size(inst: Instance, S: int) -> int:
    return int(load().ubqp_ascent_workspace_size(inst.handle, S))


def ascent(inst: Instance, X: torch.Tensor, f: torch.Tensor, idx: torch.Tensor,
           count: torch.Tensor, max_flips: int = 0, flips: torch.Tensor | None = None,
           ws: torch.Tensor | None = None, use_ws: bool = True,
           stream=None) -> torch.Tensor | None:
    """Steepest ascent of X[idx[:count]] in place.  With use_ws (default) a
    workspace is allocated if none is given, so the start-up runs on the tensor
    cores; use_ws=False selects the CUDA-core start-up."""
    S = X.shape[0]
    if ws is None and use_ws:
        ws = torch.empty(max(ascent_workspace_size(inst, S), 16), dtype=torch.uint8,
                         device=X.device)
    nbytes = ws.numel() if ws is not None else 0
    _check(load().ubqp_ascent(inst.handle, _ptr(X), _ptr(f), _ptr(idx), _ptr(count), S,
                              max_flips, _ptr(flips), _ptr(ws), nbytes, _stream(stream)))
    return flips


def ascent_trace(inst: Instance, X: torch.Tensor, f: torch.Tensor, idx: torch.Tensor,
                 count: torch.Tensor, ldt: int, max_flips: int = 0,
                 flips: torch.Tensor | None = None, trace: torch.Tensor | None = None,
                 ws: torch.Tensor | None = None, stream=None):
    """ubqp_ascent_trace: the ascent of X[idx[:count]] in place, with start s's
    flipped indices in order in trace[s, :min(flips[s], ldt)] (uint16 values
    held in an int16 tensor of S x ldt; read them with .view(torch.uint16) or
    numpy's .view(np.uint16)).  Returns (flips, trace)."""
    S = X.shape[0]
    if flips is None:
        flips = torch.zeros(S, dtype=torch.int32, device=X.device)
    if trace is None:
        trace = torch.zeros((S, ldt), dtype=torch.int16, device=X.device)
    if ws is None:
        ws = torch.empty(max(ascent_workspace_size(inst, S), 16), dtype=torch.uint8,
                         device=X.device)
    _check(load().ubqp_ascent_trace(inst.handle, _ptr(X), _ptr(f), _ptr(idx), _ptr(count), S,
                                    max_flips, _ptr(flips), _ptr(trace), ldt, _ptr(ws),
                                    ws.numel(), _stream(stream)))
    return flips, trace


def relink_workspace_size(inst: Instance, P: int, tensor_startup: bool = True) -> int:
    return int(load().ubqp_relink_workspace_size(inst.handle, P, 1 if tensor_startup else 0))


def relink(inst: Instance, X: torch.Tensor, f: torch.Tensor, G: torch.Tensor,
           tensor_startup: bool = True, ws: torch.Tensor | None = None, stream=None):
    """Path relinking of the pairs (X[p], G[p]) (ubqp_relink); f[p] = f(X[p]).
    Returns (X_best, f_best, dist)."""
    P = X.shape[0]
    Xb = torch.empty_like(X)
    fb = torch.empty(P, dtype=torch.int64, device=X.device)
    dist = torch.empty(P, dtype=torch.int32, device=X.device)
    if ws is None:
        ws = torch.empty(max(relink_workspace_size(inst, P, tensor_startup), 16),
                         dtype=torch.uint8, device=X.device)
    _check(load().ubqp_relink(inst.handle, _ptr(X), _ptr(f), _ptr(G), P, _ptr(Xb), _ptr(fb),
                              _ptr(dist), _ptr(ws), ws.numel(), _stream(stream)))
    return Xb, fb, dist


def selftest_timeout(limit_us: int = 20000, stream=None) -> int:
    """Run the bounded-wait self-test; returns its status (UBQP_ERR_TIMEOUT = -6
    when the wait gave up as it should)."""
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    return int(load().ubqp_selftest_timeout(limit_us, _ptr(st), _stream(stream)))


def best(f: torch.Tensor, X: torch.Tensor, stream=None):
    bx = torch.empty(X.shape[1], dtype=torch.int64, device=X.device)
    bf = torch.empty(2, dtype=torch.int64, device=X.device)
    _check(load().ubqp_best(_ptr(f), _ptr(X), f.shape[0], X.shape[1], _ptr(bx), _ptr(bf),
                            _stream(stream)))
    return bx, bf


def make_params(S: int, lam: float, max_flips: int = 0, mode: int = DIVERSIFY, seed: int = 0,
                round_: int = 0, div_H: int = 64, eval_path: int = EVAL_AUTO) -> Params:
    return Params(S, float(lam), max_flips, mode, seed % 2**64, round_, div_H, eval_path)


def solve_workspace_size(inst: Instance, params: Params) -> int:
    return int(load().ubqp_solve_workspace_size(inst.handle, ctypes.byref(params)))


def solve(inst: Instance, params: Params, ws: torch.Tensor | None = None,
          best_x: torch.Tensor | None = None, best_f: torch.Tensor | None = None,
          want_stats: bool = True, stream=None):
    """One round (Fig. 2's loop body over a batch).  Returns (best_x, best_f[2], stats)."""
    need = solve_workspace_size(inst, params)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=inst.device)
    bx = best_x if best_x is not None else torch.empty(inst.words, dtype=torch.int64,
                                                       device=inst.device)
    bf = best_f if best_f is not None else torch.empty(2, dtype=torch.int64, device=inst.device)
    st = Stats() if want_stats else None
    _check(load().ubqp_solve(inst.handle, ctypes.byref(params), _ptr(bx), _ptr(bf),
                             ctypes.byref(st) if st is not None else None, _ptr(ws),
                             ws.numel(), _stream(stream)))
    return bx, bf, (st.as_dict() if st is not None else None)


def solve_rounds_workspace_size(inst: Instance, params: Params, R: int) -> int:
    return int(load().ubqp_solve_rounds_workspace_size(inst.handle, ctypes.byref(params), R))


def solve_rounds(inst: Instance, params: Params, R: int, ws: torch.Tensor | None = None,
                 best_x: torch.Tensor | None = None, best_f: torch.Tensor | None = None,
                 stream=None):
    """R independent rounds run together (ubqp_solve_rounds): round k equals
    solve() with seed + k and round + k.  Returns (best_x (R, W), best_f (R, 2))."""
    dev = inst.device
    if ws is None:
        ws = torch.empty(max(solve_rounds_workspace_size(inst, params, R), 16),
                         dtype=torch.uint8, device=dev)
    if best_x is None:
        best_x = torch.empty((R, inst.words), dtype=torch.int64, device=dev)
    if best_f is None:
        best_f = torch.empty((R, 2), dtype=torch.int64, device=dev)
    _check(load().ubqp_solve_rounds(inst.handle, ctypes.byref(params), R, _ptr(best_x),
                                    _ptr(best_f), _ptr(ws), ws.numel(), _stream(stream)))
    return best_x, best_f


def search(inst: Instance, num_samples: int, starts_per_round: int, rounds: int, lam: float,
           max_flips: int = 0, seed: int = 0, div_H: int = 64, eval_path: int = EVAL_AUTO,
           stream=None) -> dict:
    """The multi-round search of Fig. 2 (ubqp_search); returns device tensors."""
    p = SearchParams(num_samples, starts_per_round, rounds, max_flips, float(lam),
                     seed % 2**64, div_H, eval_path)
    need = int(load().ubqp_search_workspace_size(inst.handle, ctypes.byref(p)))
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device=inst.device)
    bx = torch.empty(inst.words, dtype=torch.int64, device=inst.device)
    bf = torch.empty(1, dtype=torch.int64, device=inst.device)
    hist = torch.empty(max(rounds, 1), dtype=torch.int64, device=inst.device)
    st = torch.empty(3, dtype=torch.int64, device=inst.device)
    _check(load().ubqp_search(inst.handle, ctypes.byref(p), _ptr(bx), _ptr(bf), _ptr(hist),
                              _ptr(st), _ptr(ws), ws.numel(), _stream(stream)))
    return {"best_x": bx, "best_f": bf, "history": hist[:rounds], "stats": st}


def search_resume(inst: Instance, state: dict, first_round: int, num_samples: int,
                  starts_per_round: int, rounds: int, lam: float, max_flips: int = 0,
                  seed: int = 0, div_H: int = 64, eval_path: int = EVAL_AUTO,
                  stream=None) -> dict:
    """Continue a search from `state` (the dict search or search_resume
    returned) with rounds first_round .. first_round + rounds - 1
    (ubqp_search_resume); returns the new state."""
    p = SearchParams(num_samples, starts_per_round, rounds, max_flips, float(lam),
                     seed % 2**64, div_H, eval_path)
    need = int(load().ubqp_search_workspace_size(inst.handle, ctypes.byref(p)))
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device=inst.device)
    bx, bf, st = state["best_x"].clone(), state["best_f"].clone(), state["stats"].clone()
    hist = torch.empty(max(rounds, 1), dtype=torch.int64, device=inst.device)
    _check(load().ubqp_search_resume(inst.handle, ctypes.byref(p), first_round, _ptr(bx),
                                     _ptr(bf), _ptr(hist), _ptr(st), _ptr(ws), ws.numel(),
                                     _stream(stream)))
    return {"best_x": bx, "best_f": bf, "history": hist[:rounds], "stats": st}


class Batch:
    """A batch plan over prepared instances (ubqp_batch_*): one round for every
    instance per run, identical per instance to ``solve``."""

    def __init__(self, instances: list, params: Params):
        self.instances = list(instances)  # keep the handles alive
        arr = (ctypes.c_void_p * len(self.instances))(*[i.handle.value for i in self.instances])
        h = ctypes.c_void_p()
        _check(load().ubqp_batch_create(arr, len(self.instances), ctypes.byref(params),
                                        ctypes.byref(h)))
        self._h = h
        self.device = self.instances[0].device

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().ubqp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seed: int, stream=None):
        _check(load().ubqp_batch_run(self._h, seed % 2**64, _stream(stream)))

    def tune(self, stream=None):
        _check(load().ubqp_batch_tune(self._h, _stream(stream)))

    def set(self, asc_threads: int, asc_chunks: int, packed: bool = False, eval_kch: int = 16,
            eval_merged: bool = False):
        """Pin the configuration (ubqp_batch_set) instead of tuning it."""
        _check(load().ubqp_batch_set(self._h, asc_threads, asc_chunks, int(packed), eval_kch,
                                     int(eval_merged)))

    def capture(self, stream=None):
        _check(load().ubqp_batch_capture(self._h, _stream(stream)))

    def config(self) -> dict:
        v = [ctypes.c_int32() for _ in range(5)]
        _check(load().ubqp_batch_config(self._h, *[ctypes.byref(x) for x in v]))
        out = dict(zip(["asc_threads", "asc_chunks", "eval_path", "streams", "graph"],
                       [x.value for x in v]))
        pk, kch, mg = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().ubqp_batch_schedule(self._h, ctypes.byref(pk), ctypes.byref(kch),
                                          ctypes.byref(mg)))
        out.update(packed=pk.value, eval_kch=kch.value, eval_merged=mg.value)
        return out

    def result(self, i: int, stream=None):
        """(best_x words, {value, index}) of instance i, copied to new tensors."""
        W = self.instances[i].words
        bx = torch.empty(W, dtype=torch.int64, device=self.device)
        bf = torch.empty(2, dtype=torch.int64, device=self.device)
        _check(load().ubqp_batch_get(self._h, i, _ptr(bx), _ptr(bf), _stream(stream)))
        return bx, bf


class Server:
    """The request loop (ubqp_server_*): submit host instances, wait for results."""

    def __init__(self, workers: int, max_n: int, params: Params, memory_budget: int = 0,
                 max_batch: int = 0):
        """workers: lanes (concurrent batches); max_batch: requests per batch
        (0 = 16)."""
        cfg = ServerConfig(workers, max_n, memory_budget, params, max_batch)
        h = ctypes.c_void_p()
        _check(load().ubqp_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}  # host buffers of in-flight requests

    def request_bytes(self, n: int) -> int:
        return int(load().ubqp_server_request_bytes(self._h, n))

    def inject_alloc_failures(self, count: int):
        """Fault injection: the next `count` admissions fail as out of memory."""
        _check(load().ubqp_server_inject_alloc_failures(self._h, count))

    def submit(self, Q, seed: int, n: int | None = None, offset: int = 0) -> int:
        """Q: a host int8 array or CPU tensor (rows x ldq), kept alive until
        wait().  With n (and offset) the request's instance is the principal
        submatrix Q[offset:offset+n, offset:offset+n], passed in place (row
        stride ldq, no copy)."""
        import numpy as _np
        if isinstance(Q, torch.Tensor):
            assert Q.dtype == torch.int8 and Q.dim() == 2 and Q.stride(1) == 1
            ptr, rows, ldq = Q.data_ptr(), Q.shape[0], Q.stride(0)
        else:
            Q = _np.ascontiguousarray(Q, dtype=_np.int8)
            ptr, (rows, ldq) = Q.ctypes.data, Q.shape
        n = rows if n is None else int(n)
        if offset < 0 or offset + n > min(rows, ldq):
            raise ValueError("principal submatrix outside Q")
        ptr += offset * ldq + offset
        t = ctypes.c_int64()
        _check(load().ubqp_server_submit(self._h, ctypes.c_void_p(ptr), n, ldq, seed % 2**64,
                                         ctypes.byref(t)))
        self._keep[t.value] = (Q, n)
        return t.value

    def stats(self) -> dict:
        """Batches run so far, the requests they held, the largest batch."""
        v = [ctypes.c_int64() for _ in range(3)]
        _check(load().ubqp_server_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["batches", "requests", "largest"], [x.value for x in v]))

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        _check(load().ubqp_server_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int):
        """(best_f {value, index} as a list, best_x numpy uint64 words, latency s)."""
        import numpy as _np
        _, n = self._keep[ticket]
        bx = _np.zeros((n + 63) // 64, _np.uint64)
        bf = _np.zeros(2, _np.int64)
        lat = ctypes.c_double()
        try:
            _check(load().ubqp_server_wait(self._h, ticket, ctypes.c_void_p(bf.ctypes.data),
                                           ctypes.c_void_p(bx.ctypes.data), ctypes.byref(lat)))
        finally:
            self._keep.pop(ticket, None)
        return bf.tolist(), bx, lat.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().ubqp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks(l2_bytes: int = 64 << 20, reps: int = 20, int_iters: int = 50_000) -> dict:
    """The ascent's roofline rates on the current device (ubqp_peak_*), timed
    with CUDA events after one untimed warm-up launch each: L2 read GB/s over
    an L2-resident buffer, the int32 multiply-add rate and the ascent's
    element-update rate in Tops/s."""
    lib = load()
    dev = torch.cuda.current_device()
    buf = torch.zeros(l2_bytes, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream()

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    s = timed(lambda: _check(lib.ubqp_peak_l2_read(_ptr(buf), l2_bytes, reps, _ptr(sink),
                                                   _stream())))
    out = {"l2_read_gbs": l2_bytes // 16 * 16 * reps / s / 1e9, "l2_buffer_bytes": l2_bytes}
    for kind, key in ((0, "int32_imad_tops"), (1, "ascent_update_tops")):
        s = timed(lambda: _check(lib.ubqp_peak_int32(kind, int_iters, _ptr(sink), _stream())))
        out[key] = lib.ubqp_peak_int32_ops(kind, int_iters) / s / 1e12
    return out
