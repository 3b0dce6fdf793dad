"""The multi-rank path of bench.py on the CPU: two gloo ranks (one process
each) agree on the slowest rank's time and the whole-job rate, and each rank
binds its own seeded stencil (independent replicas, no data-path exchange)."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    rate = bench.job_throughput(world, 1000, 4, ms / 1000.0)
    w = workloads.config2(rank, planted=True, W=64, H=64, K=4)
    out[rank] = (ms, rate, w.text)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == 2 * 1000 * 4 / 0.015
    assert res[0][2] != res[1][2]  # each rank checks its own seeded stencil


def test_one_rank_keeps_its_own_numbers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 10, 2, 0.5) == 40.0
