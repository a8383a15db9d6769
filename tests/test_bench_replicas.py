"""The multi-GPU path of bench.py runs independent replicas (the simulator does
not shard without a per-cycle halo exchange): the job time is the slowest
rank's and the throughput counts every rank's work.  Checked with two gloo
ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.replica_throughput(100.0 * (rank + 1), 1000, world)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == (200.0, 1000 * 2 / 0.2)


def test_single_rank_is_unchanged():
    import bench
    assert bench.replica_throughput(50.0, 10, 1) == (50.0, 10 / 0.05)
