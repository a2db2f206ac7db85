"""Sharding the path range over ranks (CPU, gloo, world size 2).

Paths are keyed by their global index, so each rank integrates a disjoint
slice of every level and one all-reduce of the per-level FP64 sums gives
the single-process result -- the only exchange the multi-GPU path needs.
The ranks here run the oracle; the same split drives bench.py --gpus N.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, reqs, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = O.make_params(W.bl600(O.GL))
    rows = []
    for level, n in reqs:
        share = n // world
        first = rank * share
        cnt = share if rank < world - 1 else n - first
        s = O.level_sums(p, O.GL, level, cnt, first, 3, threads=2)
        rows.append(np.concatenate([[s["n"], s["n_nonfinite"]], s["sum"].ravel()]))
    t = torch.tensor(np.array(rows), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_reduce_to_the_single_process_sums(tmp_path):
    reqs = [(0, 20000), (2, 6001), (4, 3000)]
    out = str(tmp_path / "sums.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), reqs, out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    p = O.make_params(W.bl600(O.GL))
    for row, (level, n) in zip(got, reqs):
        s = O.level_sums(p, O.GL, level, n, 0, 3, threads=2)
        assert row[0] == s["n"] and row[1] == s["n_nonfinite"]
        assert np.allclose(row[2:], s["sum"].ravel(), rtol=1e-12, atol=1e-9)
