"""The multi-process host logic of bench.py on CPU, two gloo ranks.

* The whole job's time is its slowest rank's: `_max_over_ranks` gives every
  rank the maximum.
* A batch split over ranks: `_rank_share` (the library's LPT plan with one
  chain per rank) gives each problem to exactly one rank, with no collective
  in the data path, and the ranks' loads differ by at most the largest cost.
"""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

COSTS = [7.0, 3.5, 9.25, 1.0, 4.0, 4.0, 8.5, 2.25, 6.0, 5.5, 0.75]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        mx = bench._max_over_ranks(1.5 + rank, ws, device="cpu")
        share = bench._rank_share(COSTS, ws, rank)
        gathered = [None] * ws
        dist.all_gather_object(gathered, share)
        out[rank] = (mx, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        mx, shares = res[rank]
        assert mx == 1.5 + (ws - 1)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(COSTS)))  # every problem on exactly one rank
        loads = [sum(COSTS[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(COSTS)
    assert res[0][1] == res[1][1]  # both ranks computed the same plan


def test_one_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(2.5, 1) == 2.5
    assert bench._rank_share(COSTS, 1, 0) == list(range(len(COSTS)))
