"""The multi-GPU path of bench.py on the host, as two gloo ranks on the CPU:
every rank solves its own units (round-robin shards of a batch, or its own
seeded cell), and the only exchange is the timing reduction (max of the
ranks' milliseconds, sum of their iterations) between barriers."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms, its = bench.aggregate(10.0 + 5.0 * rank, 13 + rank, world)
        units = bench.shard(64, rank, world)
        case = bench.make_workload("cube8", rank)
        ce = np.asarray(case["state"]["ce"], dtype=float)
        bench.barrier(world)
        q.put((rank, ms, its, units, float(ce.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, it0, u0, ce0), (r1, ms1, it1, u1, ce1) = out
    assert (r0, r1) == (0, 1)
    assert ms0 == ms1 == 15.0                        # max over ranks
    assert it0 == it1 == 27.0                        # sum over ranks
    assert sorted(u0 + u1) == list(range(64)) and not set(u0) & set(u1)
    assert ce0 != ce1                                # each rank its own seeded cell


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 13, 1) == (12.5, 13)
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.make_workload("cube8", 0)["state"].keys() == bench.make_workload("cube8", 1)["state"].keys()
