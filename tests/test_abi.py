"""The C-ABI library builds, loads without a GPU, exports every declared symbol,
and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1706_00037_gb300 import ubqp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "ubqp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ubqp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ubqp_diversify", "ubqp_eval", "ubqp_screen", "ubqp_ascent", "ubqp_solve",
              "ubqp_q_prepare", "ubqp_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ubqp.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ubqp.EXPORTS) <= set(declared_functions())


def test_strerror_and_version():
    lib = ubqp.load()
    assert lib.ubqp_abi_version() == 5
    for st, name in ubqp.STATUS_NAMES.items():
        assert lib.ubqp_strerror(st)
    assert lib.ubqp_strerror(0) == b"ok"


def test_host_side_argument_errors():
    lib = ubqp.load()
    h = ctypes.c_void_p()
    # NULL Q, bad n, NULL out: rejected before any CUDA call
    assert lib.ubqp_q_prepare(None, 10, 10, None, ctypes.byref(h)) == -1
    assert lib.ubqp_q_prepare(ctypes.c_void_p(16), 0, 10, None, ctypes.byref(h)) == -7
    assert lib.ubqp_q_prepare(ctypes.c_void_p(16), 10, 5, None, ctypes.byref(h)) == -1
    assert lib.ubqp_q_prepare(ctypes.c_void_p(16), 10, 10, None, None) == -1
    assert b"out" in lib.ubqp_last_error()
    assert lib.ubqp_q_prepare_into_async(ctypes.c_void_p(16), 10, 10, None, 0, None,
                                         ctypes.byref(h)) == -1
    assert b"arena" in lib.ubqp_last_error()
    assert lib.ubqp_screen(None, 10, 0.5, None, None, None, None, None) == -1
    p = ubqp.Params(0, 0.5, 0, 1, 0, 0, 64, 0)
    assert lib.ubqp_solve(None, ctypes.byref(p), None, None, None, None, 0, None) == -1
    assert lib.ubqp_eval_workspace_size(None, 10, 0) == 0
    assert lib.ubqp_q_info(None, None, None, None, None, None) == -1
    assert lib.ubqp_ascent_trace(None, None, None, None, None, 1, 0, None, None, 4, None, 0,
                                 None) == -1
    assert b"trace" in lib.ubqp_last_error()
    assert lib.ubqp_solve_rounds(None, ctypes.byref(p), 2, None, None, None, 0, None) == -1
    assert lib.ubqp_solve_rounds_workspace_size(None, ctypes.byref(p), 2) == 0
    lib.ubqp_q_destroy(None)  # no-op
    # relinking, search, batch plans and the server validate on the host too
    assert lib.ubqp_relink(None, None, None, None, 4, None, None, None, None, 0, None) == -1
    assert lib.ubqp_relink_workspace_size(None, 4, 1) == 0
    sp = ubqp.SearchParams(100, 10, 2, 0, 0.5, 1, 64, 0)
    assert lib.ubqp_search(None, ctypes.byref(sp), None, None, None, None, None, 0, None) == -1
    b = ctypes.c_void_p()
    assert lib.ubqp_batch_create(None, 1, ctypes.byref(p), ctypes.byref(b)) == -1
    assert lib.ubqp_batch_create(None, 1, ctypes.byref(p), None) == -1
    srv = ctypes.c_void_p()
    assert lib.ubqp_server_create(None, ctypes.byref(srv)) == -1
    assert lib.ubqp_server_create(None, None) == -1
    assert lib.ubqp_server_request_bytes(None, 100) == 0
    lib.ubqp_server_destroy(None)  # no-op
    lib.ubqp_batch_destroy(None)  # no-op


def test_params_layout_matches_header():
    # ubqp_params: int64, double, int32, int32, uint64, uint64, int32, int32
    assert ctypes.sizeof(ubqp.Params) == 48
    assert ctypes.sizeof(ubqp.Stats) == 64


def test_binding_refuses_pageable_host_q():
    """The binding takes Q on the device or in pinned host memory only."""
    import torch
    Q = torch.zeros((8, 8), dtype=torch.int8)
    with pytest.raises(ValueError):
        ubqp.Instance(Q)
    with pytest.raises(ValueError):
        ubqp.Instance(torch.zeros((8, 8), dtype=torch.int16))
