"""The allocation-free batched launch (GPU).

``mlmc_multilevel_sums_noalloc`` serves callers that may not allocate device
memory (a framework whose pool owns all of it, a loop that must never block
in cudaMalloc); its scratch is a static device array inside the library.  It
is called here through the C ABI, twice in a row with different batches, and
each result is checked against the workspace-based ``mlmc_multilevel_sums``:
both forms split a batch that fits the array into the same work items, so
the results must be bit-identical (counts and FP64 sums).  The second call
must not see anything the first left in the shared array.  Adaptive-timestep
and FP64 batches take other branches of the planner and kernels and are
checked the same way.  After a warm-up call, repeated calls must leave the
device's free memory unchanged.  This file is collected last so a failure
here stops a run only after every other test has run; it also passes alone
in a fresh process.
"""
import ctypes as C

import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fn():
    fn = G.lib().mlmc_multilevel_sums_noalloc
    fn.argtypes = [C.POINTER(G.LevelRequest), C.c_int, C.c_int, C.POINTER(G.Params),
                   C.c_uint64, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def _reqs(reqs):
    arr = (G.LevelRequest * len(reqs))()
    for k, (lvl, first, count) in enumerate(reqs):
        arr[k].level, arr[k].first, arr[k].count = lvl, first, count
    return arr


def _noalloc(reqs, integ, params, seed, stream, d_out=None):
    import torch
    n = len(reqs)
    if d_out is None:
        d_out = torch.zeros(n * C.sizeof(G.LevelResult), dtype=torch.uint8, device="cuda")
    rc = _fn()(_reqs(reqs), n, integ, C.byref(params), seed, C.c_void_p(stream.cuda_stream),
               C.c_void_p(d_out.data_ptr()))
    assert rc == G.OK, G.strerror(rc)
    stream.synchronize()
    out = (G.LevelResult * n).from_buffer_copy(d_out.cpu().numpy().tobytes())
    return [G._level_result(out[k]) for k in range(n)]


def _check_batches(batches, integ, params, seed):
    import torch
    stream = torch.cuda.current_stream()
    for reqs in batches:
        got = _noalloc(reqs, integ, params, seed, stream)
        ref = G.multilevel_sums(reqs, integ, params, seed)
        assert len(got) == len(ref)
        for a, b in zip(got, ref):
            assert a == b                          # same items: bit-identical sums
        assert all(g["n"] + g["n_nonfinite"] == c for g, (_, _, c) in zip(got, reqs))


def test_noalloc_launch_matches_workspace_launch_twice_in_a_row():
    params = G.make_params(W.bl600(G.BAOAB), precision=G.FP32)
    first = [(6, 0, 30001), (4, 5, 60000), (2, 0, 250000), (0, 11, 1000000)]
    second = [(9, 3, 2000), (1, 0, 400001)]
    _check_batches((first, second), G.BAOAB, params, 7)


def test_noalloc_fp64_batch_matches_workspace_launch():
    params = G.make_params(W.bl600(G.GL), precision=G.FP64)
    _check_batches(([(5, 0, 3001), (2, 100, 20000), (0, 0, 70001)], [(3, 7, 5000)]),
                   G.GL, params, 11)


def test_noalloc_adaptive_batch_matches_workspace_launch():
    params = G.make_params(dict(W.PAPER, z_adapt=0.05), precision=G.FP32)
    _check_batches(([(4, 0, 3001), (2, 9, 20000), (0, 0, 40001)], [(5, 1, 1000)]),
                   G.SE, params, 5)


def test_noalloc_calls_leave_free_device_memory_unchanged():
    import torch
    stream = torch.cuda.current_stream()
    params = G.make_params(W.bl600(G.BAOAB), precision=G.FP32)
    reqs = [(5, 0, 20000), (1, 0, 300000)]
    d_out = torch.zeros(len(reqs) * C.sizeof(G.LevelResult), dtype=torch.uint8, device="cuda")
    _noalloc(reqs, G.BAOAB, params, 3, stream, d_out)    # warm-up: module loading
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in range(4, 9):
        _noalloc(reqs, G.BAOAB, params, seed, stream, d_out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_out_of_order_and_oversized_batches():
    import torch
    stream = torch.cuda.current_stream()
    params = G.make_params(W.bl600(G.GL))
    fn = _fn()
    d_out = torch.zeros(64 * C.sizeof(G.LevelResult), dtype=torch.uint8, device="cuda")
    arr = _reqs([(0, 0, 10)] * 33)
    assert fn(arr, 33, G.GL, C.byref(params), 1, C.c_void_p(stream.cuda_stream),
              C.c_void_p(d_out.data_ptr())) == G.EINVAL
    arr[0].level, arr[1].level = 1, 2                     # finer level after a coarser one
    assert fn(arr, 2, G.GL, C.byref(params), 1, C.c_void_p(stream.cuda_stream),
              C.c_void_p(d_out.data_ptr())) == G.EINVAL
