"""The replica host logic on two CPU ranks (gloo): distinct seeds per rank, and the job's
throughput as all ranks' updates over the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2212_11878_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r advances (r + 1) * 1e6 particle updates in (r + 1) * 10 ms
        value, ms, total = replicas.job_throughput((rank + 1) * 1e6, (rank + 1) * 10.0, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, (replicas.box_seed(7, rank), replicas.ensemble_seed(7, rank)))
        out[rank] = (value, ms, total, seeds)
    finally:
        dist.destroy_process_group()


def test_two_rank_throughput_and_seeds():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        value, ms, total, seeds = res[rank]
        assert ms == 20.0                      # the slowest rank's time
        assert total == 3e6                    # all ranks' updates
        assert value == pytest.approx(3e6 / 0.020)
        assert len({s[0] for s in seeds}) == world and len({s[1] for s in seeds}) == world


def test_single_process_is_plain_rate():
    value, ms, total = replicas.job_throughput(5e6, 10.0, None)
    assert value == pytest.approx(5e8) and ms == 10.0 and total == 5e6
