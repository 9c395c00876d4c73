"""The multi-process (N > 1) host logic of bench.py on CPU ranks (gloo, world size 2).

Replicas share nothing on the data path; what ranks do together is the barrier around
the timed region, the max over ranks of the elapsed time, the whole-job rate from it,
and the split of an independent batch of instances.  Each is checked here on two CPU
processes rendezvousing on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t = 1.5 + rank                       # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, world, device="cpu")
        rate = bench.whole_job_rate(64, tmax, world)
        mine = bench.shard(257, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        bench.barrier(world)
        q.put((rank, tmax, rate, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate, gathered in out:
        assert tmax == 2.5                   # the slowest rank's time on every rank
        assert rate == pytest.approx(64 * 2 / 2.5)
        allitems = sorted(i for part in gathered for i in part)
        assert allitems == list(range(257))  # disjoint and complete
        assert abs(len(gathered[0]) - len(gathered[1])) <= 1
