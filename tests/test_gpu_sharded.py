"""The adaptive estimator sharded over ranks (mlmc_estimate_sharded) on one
GPU: each rank integrates its slice of every level and one all-reduce per
pass combines the per-level sums.  The ranks' kernels never wait on each
other; only the hosts meet in the reduction.

* two ranks as threads (reduction through a host barrier) and two ranks as
  processes (torch.distributed gloo) both return the single-process result:
  the same levels and sample counts, estimates equal to FP64 rounding;
* a rank whose launch fails still joins the reduction, so every rank
  returns an error instead of waiting;
* a reduce hook that fails gives MLMC_ECOMM;
* with FP64 paths the two gloo ranks' sample counts equal the FP64 oracle
  driver's and their estimate equals its estimate to 1e-10: the all-reduce
  of the per-level sums preserves the telescoping estimator (Eqs.
  telescoping_sum and Yhatell) whatever the split.
"""
import os
import socket
import threading

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

pytestmark = pytest.mark.gpu

EPS = 2e-3 * 600


def _params(precision=G.FP32):
    return G.make_params(W.bl600(G.GL, n_init=5000, L_max=8), precision=precision)


class HostSum:
    """All-reduce of W threads through a barrier (for ranks in one process)."""

    def __init__(self, world, timeout=60.0):
        self.world = world
        self.bar = threading.Barrier(world, timeout=timeout)
        self.parts = [None] * world
        self.total = None

    def hook(self, rank):
        def reduce(values):
            self.parts[rank] = np.array(values)
            if self.bar.wait() == 0:
                self.total = sum(self.parts)
            self.bar.wait()
            return list(self.total)
        return reduce


def _run_threads(world, make_args):
    out = [None] * world

    def run(rank):
        try:
            out[rank] = make_args(rank)()
        except Exception as e:             # noqa: BLE001 -- the test inspects it
            out[rank] = e
    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in ts), "a rank did not finish"
    return out


def _same_result(a, b):
    assert a["L"] == b["L"] and a["N"] == b["N"], (a["L"], b["L"], a["N"], b["N"])
    assert a["total_path_steps"] == b["total_path_steps"]
    for q in range(2):
        assert a["estimate"][q] == pytest.approx(b["estimate"][q], rel=1e-12, abs=1e-12)


def test_two_thread_ranks_give_the_single_process_result():
    ref = G.estimate(EPS, G.GL, _params(), 13)
    hs = HostSum(2)

    def make(rank):
        p = _params()
        ws = G.Workspace(p)
        st = torch.cuda.Stream()
        return lambda: G.estimate_sharded(EPS, G.GL, p, 13, rank, 2, hs.hook(rank),
                                          workspace=ws, stream=st)
    res = _run_threads(2, make)
    for r in res:
        assert isinstance(r, dict), r
        _same_result(r, ref)
    assert res[0]["estimate"] == res[1]["estimate"]


def test_a_failing_rank_stops_every_rank():
    hs = HostSum(2)

    def make(rank):
        p = _params()
        ws = G.Workspace(p)
        if rank == 1:
            ws.nbytes = 256                # far too small: this rank's launches fail
        st = torch.cuda.Stream()
        return lambda: G.estimate_sharded(EPS, G.GL, p, 13, rank, 2, hs.hook(rank),
                                          workspace=ws, stream=st)
    res = _run_threads(2, make)
    assert isinstance(res[0], G.MLMCError) and res[0].code == G.ECOMM
    assert isinstance(res[1], G.MLMCError) and res[1].code == G.EWORKSPACE


def test_a_failing_reduction_is_reported():
    def bad(values):
        raise RuntimeError("link down")
    with pytest.raises(G.MLMCError) as e:
        G.estimate_sharded(EPS, G.GL, _params(), 13, 0, 2, bad)
    assert e.value.code == G.ECOMM


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _proc(rank, world, port, out_path, precision=G.FP32):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    r = G.estimate_sharded(EPS, G.GL, _params(precision), 13, rank, world, G.torch_allreduce())
    np.save(out_path + "_%d.npy" % rank,
            np.array([r["L"]] + r["N"] + list(r["estimate"]) + [r["total_path_steps"]],
                     dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_process_ranks_over_gloo_give_the_single_process_result(tmp_path):
    out = str(tmp_path / "res")
    mp.start_processes(_proc, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    ref = G.estimate(EPS, G.GL, _params(), 13)
    want = np.array([ref["L"]] + ref["N"] + list(ref["estimate"]) + [ref["total_path_steps"]],
                    dtype=np.float64)
    for rank in range(2):
        got = np.load(out + "_%d.npy" % rank)
        assert got.shape == want.shape
        n = 1 + len(ref["N"])
        assert np.array_equal(got[:n], want[:n])
        assert np.allclose(got[n:n + 2], want[n:n + 2], rtol=1e-12, atol=1e-12)
        assert got[-1] == want[-1]


def test_two_process_fp64_ranks_over_gloo_equal_the_oracle_driver(tmp_path):
    out = str(tmp_path / "res64")
    mp.start_processes(_proc, args=(2, _free_port(), out, G.FP64), nprocs=2, join=True,
                       start_method="spawn")
    po = O.make_params(W.bl600(G.GL, n_init=5000, L_max=8), uniform_map=O.U32)
    o = O.estimate(po, O.GL, EPS, seed=13)
    assert o["converged"] == 1
    for rank in range(2):
        got = np.load(out + "_%d.npy" % rank)
        L = int(got[0])
        n = 1 + (L - po.level_min + 1)
        assert L == o["L"]
        assert [int(x) for x in got[1:n]] == o["N"]
        assert got[n] == pytest.approx(o["estimate"][0], rel=1e-10)
        assert got[n + 1] == pytest.approx(o["estimate"][1], rel=1e-10, abs=1e-12)
        assert int(got[-1]) == o["total_path_steps"]
