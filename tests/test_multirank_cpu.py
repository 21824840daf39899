"""The N > 1 path on the CPU with world_size-2 gloo ranks: each rank runs its own seeded
workload (weak scaling, no collective on the data path), a design map is sharded
without overlap, and the job time is the maximum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_22308_gb300 import workloads as W
    mine = W.rank_workload("md_janus_512", rank)
    dm = W.shard(W.design_map_256(4, 10), rank, world)
    t = bench.max_over_ranks(1.5 + rank, dist)
    q.put((rank, [i["eps1"] for i in mine], [round(i["eps2"], 12) for i in dm], t))
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, eps0, dm0, t0), (r1, eps1, dm1, t1) = out
    assert eps0 != eps1                      # distinct seeded problems per rank
    assert t0 == t1 == 2.5                   # both ranks see the slowest rank's time
    from paper_2509_22308_gb300 import workloads as W
    full = [round(i["eps2"], 12) for i in W.design_map_256(4, 10)]
    assert sorted(dm0 + dm1) == sorted(full) and not set(dm0) & set(dm1)
