"""The allocation-free batched launch (GPU).

``mlmc_multilevel_sums_noalloc`` serves callers that may not allocate device
memory (a framework whose pool owns all of it, a loop that must never block
in cudaMalloc); its scratch is a static device array inside the library.  It
is called here through the C ABI, twice in a row with different batches, and
each result is checked against the workspace-based ``mlmc_multilevel_sums``
with the tolerance of the other batched-launch tests: counts exact, FP64 sums
to 1e-11 relative.  The second call must not see anything the first left in
the shared array.  This file is collected last so a failure here stops a run
only after every other test has run; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(reqs, integ, params, seed, stream):
    import torch
    L = G.lib()
    fn = L.mlmc_multilevel_sums_noalloc
    fn.argtypes = [C.POINTER(G.LevelRequest), C.c_int, C.c_int, C.POINTER(G.Params),
                   C.c_uint64, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    n = len(reqs)
    arr = (G.LevelRequest * n)()
    for k, (lvl, first, count) in enumerate(reqs):
        arr[k].level, arr[k].first, arr[k].count = lvl, first, count
    d_out = torch.zeros(n * C.sizeof(G.LevelResult), dtype=torch.uint8, device="cuda")
    rc = fn(arr, n, integ, C.byref(params), seed, C.c_void_p(stream.cuda_stream),
            C.c_void_p(d_out.data_ptr()))
    assert rc == G.OK, G.strerror(rc)
    stream.synchronize()
    out = (G.LevelResult * n).from_buffer_copy(d_out.cpu().numpy().tobytes())
    return [G._level_result(out[k]) for k in range(n)]


def _same(a, b):
    assert a["n"] == b["n"] and a["n_nonfinite"] == b["n_nonfinite"]
    assert a["path_steps"] == b["path_steps"]
    assert np.array_equal(np.array(a["sum"][1]), np.array(b["sum"][1]))
    assert np.allclose(a["sum"][0], b["sum"][0], rtol=1e-11, atol=1e-9)


def test_noalloc_launch_matches_workspace_launch_twice_in_a_row():
    import torch
    stream = torch.cuda.current_stream()
    params = G.make_params(W.bl600(G.BAOAB), precision=G.FP32)
    first = [(6, 0, 30001), (4, 5, 60000), (2, 0, 250000), (0, 11, 1000000)]
    second = [(9, 3, 2000), (1, 0, 400001)]
    for reqs in (first, second):
        got = _noalloc(reqs, G.BAOAB, params, 7, stream)
        ref = G.multilevel_sums(reqs, G.BAOAB, params, 7)
        assert len(got) == len(ref)
        for a, b in zip(got, ref):
            _same(a, b)
        assert all(g["n"] == c for g, (_, _, c) in zip(got, reqs))


def test_noalloc_rejects_out_of_order_and_oversized_batches():
    import torch
    stream = torch.cuda.current_stream()
    params = G.make_params(W.bl600(G.GL))
    L = G.lib()
    fn = L.mlmc_multilevel_sums_noalloc
    fn.argtypes = [C.POINTER(G.LevelRequest), C.c_int, C.c_int, C.POINTER(G.Params),
                   C.c_uint64, C.c_void_p, C.c_void_p]
    d_out = torch.zeros(64 * C.sizeof(G.LevelResult), dtype=torch.uint8, device="cuda")
    arr = (G.LevelRequest * 33)()
    for k in range(33):
        arr[k].level, arr[k].first, arr[k].count = 0, 0, 10
    assert fn(arr, 33, G.GL, C.byref(params), 1, C.c_void_p(stream.cuda_stream),
              C.c_void_p(d_out.data_ptr())) == G.EINVAL
    arr[0].level, arr[1].level = 1, 2                     # finer level after a coarser one
    assert fn(arr, 2, G.GL, C.byref(params), 1, C.c_void_p(stream.cuda_stream),
              C.c_void_p(d_out.data_ptr())) == G.EINVAL
