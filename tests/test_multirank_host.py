"""Host-side logic of the multi-GPU benchmark path (independent replicas,
one per rank, timed between barriers) with world_size 2 on the gloo backend.
No GPU: the replicas' step timings are faked on the host."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = [12.0, 20.0][rank]                  # the second replica is slower
    launches = [1000, 1000][rank]
    dist.barrier()
    (tmax,), (lsum,) = bench.reduce_over_ranks(dist, "cpu", [t_ms], [launches])
    value = bench.job_value(64 * 128 ** 3 * 200, world, tmax)
    out[rank] = (tmax, lsum, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_takes_slowest_time_and_sums_work():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        tmax, lsum, value = out[r]
        assert tmax == 20.0 and lsum == 2000
        assert value == pytest.approx(2 * 64 * 128 ** 3 * 200 / 0.020)


def test_single_process_passes_values_through():
    import bench
    (t,), (n,) = bench.reduce_over_ranks(None, "cpu", [3.5], [7])
    assert t == 3.5 and n == 7
    assert bench.job_value(100, 1, 1000.0) == pytest.approx(100.0)
