"""A batch split over ranks (paper_2604_02106_b300.shard) on the CPU: the
longest-processing-time partition, and two gloo ranks that each check their
share (here with the CPU oracle standing in for the GPU batch) and gather the
verdicts, which must equal a one-rank run item for item."""
import os
import random
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2604_02106_b300 import shard  # noqa: E402


def test_lpt_partition_covers_every_item_once_and_balances():
    rng = random.Random(5)
    for world in (1, 2, 3, 8):
        costs = [int(10 ** rng.uniform(3, 7)) for _ in range(200)]
        parts = shard.lpt_partition(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # list scheduling: no rank exceeds the mean load by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
        assert parts == shard.lpt_partition(costs, world)  # deterministic
    # the largest items go to different ranks first
    assert shard.lpt_partition([5, 9, 1, 9], 2) == [[0, 1], [2, 3]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _items():
    import workloads
    return workloads.config3()[:18] + [workloads.config4(i, hi_exp=4.0) for i in range(12)]


def _oracle_checker(kernels):
    import oracle
    out = []
    for k in kernels:
        w = k.workload
        o = oracle.check(w.text, w.binding, pair=False)
        out.append((o.racy, o.n_witness, o.n_by_kind, tuple(o.witnesses[:8])))
    return out


def _bound(ws):
    import paper_2604_02106_b300 as hg
    ks = []
    for w in ws:
        k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
        k.workload = w
        ks.append(k)
    return ks


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2604_02106_b300 import shard as sh
    ks = _bound(_items())
    seen = []

    def checker(share):
        seen.extend(k.workload.name for k in share)
        return _oracle_checker(share)
    res = sh.check_sharded(ks, dist=dist, checker=checker)
    out[rank] = (res, seen)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_verdicts_of_a_one_rank_run():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    ks = _bound(_items())
    alone = shard.check_sharded(ks, checker=_oracle_checker)
    assert got[0][0] == got[1][0] == alone
    # each rank checked its own share, together every item once
    assert not set(got[0][1]) & set(got[1][1])
    assert sorted(got[0][1] + got[1][1]) == sorted(k.workload.name for k in ks)
    costs = [k.info()[0] for k in ks]
    assert costs == [k.workload.binding.instances_per_access([8]) * 12 for k in ks[:18]] + costs[18:]
