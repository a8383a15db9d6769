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


def test_byte_model_of_the_measurement_plan():
    """176 B per router-cycle (8 link slots of 16 B, 2 x 24 B of core and
    queue scalars) plus one L1 set per reference, one L2 set per L1 miss and
    one L2 set (+ a directory word under LSPD) per ejected flit; on the stored
    record of the 208x208 period-10 run it is 177.8 B per router-cycle."""
    import json
    import os

    import bench
    from paper_1508_03235_b300 import inputs as I
    p = I.mesh_208(10)
    zero = {k: 0 for k in ("refs", "l1_miss", "ejected")}
    assert bench.algorithmic_bytes(zero, 1000, p) == 176 * 1000
    one = dict(zero, refs=1, l1_miss=1, ejected=1)
    assert bench.algorithmic_bytes(one, 0, p) == (8 * 4 + 8) + (8 * 16 + 8) + 8 * 16
    assert bench.algorithmic_bytes(one, 0, dict(p, policy=1)) == (8 * 4 + 8) + (8 * 16 + 8) + 8 * 16 + 4
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "full_length.json")))
    st = rec["workloads"]["mesh208_period10"]["checkpoints"][-1]["stats"]
    per = bench.algorithmic_bytes(st, 208 * 208 * 50_000, p) / (208 * 208 * 50_000)
    assert 177.7 < per < 177.9
