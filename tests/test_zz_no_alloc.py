"""The allocation-free evaluation entry point, ubqp_eval_noalloc.

Some callers cannot allocate device memory: their device memory is reserved
by another allocator (a framework's caching pool, a fixed memory budget), or
they must not run cudaMalloc/cudaFree in a latency-critical loop, since those
can synchronise the whole device.  ubqp_eval_noalloc serves them with a scratch
array built into the library.  These tests call it through the C ABI and check,
on two calls in a row, that it returns exactly what ubqp_eval (with a caller
workspace) returns, that a call changes the device's free memory by nothing,
that a request needing exactly the whole array works and one needing more is
refused.  The file is collected last so that a failure here cannot hide any
other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1706_00037_gb300 import synth, ubqp

pytestmark = pytest.mark.gpu

MAX_BYTES = 16 << 20  # UBQP_EVAL_NOALLOC_MAX_BYTES


def _noalloc(lib, inst, X, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ubqp_eval_noalloc(inst.handle, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), stream)


def _need(S, n):
    return (S + 127) // 128 * 128 * ((n + 255) // 256 * 256) * 2


@pytest.mark.parametrize("n,density,S", [(1000, 1.0, 300), (7000, 1.0, 1000),
                                         (8192, 1.0, 1000)])
def test_noalloc_eval_equals_workspace_eval_on_consecutive_calls(n, density, S):
    lib = ubqp.load()
    assert _need(S, n) <= MAX_BYTES
    Q = synth.make_instance(n, density, n)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    for seed in (101, 202):  # two calls in a row, different batches
        X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=seed)
        want = ubqp.eval(inst, X, path=ubqp.EVAL_TC)
        got = torch.full((S,), -1, dtype=torch.int64, device="cuda")
        assert _noalloc(lib, inst, X, got) == 0, lib.ubqp_last_error()
        inst.sync()
        assert torch.equal(got, want)
        if n <= 1000:  # and every value against the CPU oracle
            Xh = X.cpu().numpy().view(np.uint64)
            assert np.array_equal(got.cpu().numpy(), orc.eval(Q, Xh))


def test_noalloc_eval_exactly_fills_the_builtin_scratch():
    # 1000 starts at n = 8192: 1024 padded rows x 8192 bf16 columns = 16 MiB
    assert _need(1000, 8192) == MAX_BYTES
    lib = ubqp.load()
    n, S = 8192, 1000
    Q = synth.make_instance(n, 1.0, 5)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=7)
    want = ubqp.eval(inst, X, path=ubqp.EVAL_TC_STAGED)
    got = torch.full((S,), -1, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, inst, X, got) == 0, lib.ubqp_last_error()
    inst.sync()
    assert torch.equal(got, want)
    # 25 starts more need another 128 padded rows: refused before any work
    S1 = S + 25
    X1 = torch.zeros((S1, inst.words), dtype=torch.int64, device="cuda")
    out1 = torch.full((S1,), -1, dtype=torch.int64, device="cuda")
    assert _need(S1, n) > MAX_BYTES
    assert _noalloc(lib, inst, X1, out1) == -7
    assert b"built-in" in lib.ubqp_last_error()
    inst.sync()
    assert bool((out1 == -1).all())


def test_noalloc_eval_leaves_free_device_memory_unchanged():
    lib = ubqp.load()
    n, S = 3000, 700
    Q = synth.make_instance(n, 0.5, 9)
    inst = ubqp.Instance(torch.from_numpy(Q).cuda())
    X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=3)
    got = torch.full((S,), -1, dtype=torch.int64, device="cuda")
    want = ubqp.eval(inst, X, path=ubqp.EVAL_TC)
    # the first call may load the module (placing the static array); after it,
    # calls take no device memory at all.  Every tensor the calls write is made
    # before the first reading and compared after the second, so that nothing
    # of torch's allocator runs in between.
    assert _noalloc(lib, inst, X, got) == 0, lib.ubqp_last_error()
    outs = [torch.full((S,), -1, dtype=torch.int64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for out in outs:
        assert _noalloc(lib, inst, X, out) == 0, lib.ubqp_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for out in outs:
        assert torch.equal(out, want)
    inst.sync()


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
