"""The multi-rank bench path on CPU: two gloo ranks (spawned processes) agree
on the slowest rank's time and the whole-job rate.  Each rank runs an
independent replica, so this max-over-ranks timing is the only exchange."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    ms = bench.reduce_max(times[rank])
    dist.barrier()
    out[rank] = (ws, r, ms, bench.job_rate(1000.0, ws, ms))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_job_rate(world):
    times = [12.5, 40.0, 7.25][:world]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True)
    for rank in range(world):
        ws, r, ms, rate = out[rank]
        assert (ws, r) == (world, rank)
        assert ms == max(times)
        assert rate == pytest.approx(1000.0 * world / (max(times) / 1000.0))


def test_single_process_is_the_identity():
    assert not dist.is_initialized()
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_rate(500.0, 1, 250.0) == pytest.approx(2000.0)
