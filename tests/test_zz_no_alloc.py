"""The allocation-free evaluation entry point, ubqp_eval_noalloc.

Some callers cannot allocate device memory (their device memory is reserved by
another allocator, or they must not run cudaMalloc/cudaFree in a hot loop);
ubqp_eval_noalloc serves them with a scratch array built into the library.
This test calls it through the C ABI and checks, on two calls in a row, that
it returns exactly what ubqp_eval (with a caller workspace) returns.  The file
is collected last so that a failure here cannot hide any other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu


def _noalloc(lib, inst, X, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ubqp_eval_noalloc(inst.handle, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("n,density,S", [(1000, 1.0, 300), (7000, 1.0, 1000)])
def test_noalloc_eval_equals_workspace_eval_on_consecutive_calls(n, density, S):
    lib = ubqp.load()
    Q = synth.make_instance(n, density, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    for seed in (101, 202):  # two calls in a row, different batches
        X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=seed)
        want = ubqp.eval(inst, X, path=ubqp.EVAL_TC)
        got = torch.full((S,), -1, dtype=torch.int64, device="cuda")
        assert _noalloc(lib, inst, X, got) == 0, lib.ubqp_last_error()
        inst.sync()
        assert torch.equal(got, want)


def test_noalloc_eval_rejects_oversized_requests():
    lib = ubqp.load()
    n = 7000
    Q = synth.make_instance(n, 0.1, 1)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    S = 2000  # 2048 * 7168 * 2 bytes > the built-in scratch
    X = torch.zeros((S, inst.words), dtype=torch.int64, device="cuda")
    out = torch.zeros(S, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, inst, X, out) == -7
    assert b"built-in" in lib.ubqp_last_error()
    inst.sync()
