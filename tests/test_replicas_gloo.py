"""The replica host logic on two CPU ranks (gloo): distinct seeds per rank, the job's
throughput as all ranks' updates over the slowest rank's time, and a rank that leaves: the
other rank's next collective ends with an error instead of waiting forever."""
import datetime
import os
import socket
import time

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
    with mp.get_context("spawn").Manager() as mgr:
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


def _leaving_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        out[rank] = "left"  # leaves between steps, with no collective in flight
        return
    t0 = time.time()
    try:
        replicas.job_throughput(1e6, 10.0, dist)
        out[rank] = ("no error", time.time() - t0)
    except Exception as e:  # gloo reports the closed peer or the timeout
        out[rank] = ("error", time.time() - t0, type(e).__name__)


@pytest.mark.timeout(120)
def test_rank_that_leaves_ends_the_next_collective_with_an_error():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_leaving_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[1] == "left"
    assert res[0][0] == "error", res[0]
    assert res[0][1] < 30.0  # within the process group's timeout, with margin


def test_single_process_is_plain_rate():
    value, ms, total = replicas.job_throughput(5e6, 10.0, None)
    assert value == pytest.approx(5e8) and ms == 10.0 and total == 5e6
