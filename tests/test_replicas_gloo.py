"""Host logic of the N > 1 benchmark path (independent replicas, one per
GPU): the whole-job rate is every rank's units over the slowest rank's time,
and independent problems are split into contiguous shares.  Runs as two gloo
ranks on the CPU."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank k processed 10 (k + 1) units in k + 1 seconds
        rate, t_max = bench.whole_job_rate(dist, 10.0 * (rank + 1), float(rank + 1))
        mx = bench.max_over_ranks(dist, 3.0 - rank)
        dist.barrier()
        q.put((rank, rate, t_max, mx))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, t_max, mx in out:
        assert t_max == 2.0           # the slower rank sets the time
        assert rate == pytest.approx(30.0 / 2.0)  # all units over it
        assert mx == 3.0


def test_single_process_needs_no_group():
    assert bench.whole_job_rate(None, 12.0, 3.0) == (4.0, 3.0)
    assert bench.max_over_ranks(None, 5.0) == 5.0


@pytest.mark.parametrize("n,world", [(256, 1), (256, 2), (256, 3), (7, 8), (0, 2)])
def test_shards_partition_the_problems(n, world):
    parts = [bench.shard(n, k, world) for k in range(world)]
    flat = [i for p in parts for i in p]
    assert flat == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1
