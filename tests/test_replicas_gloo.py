"""Host logic of the N-replica benchmark on CPU processes (gloo, world size 2):
the job time is the slowest rank's, the value counts every rank's particles."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank)          # rank 1 is slower
    v = bench.job_throughput(1000, world, 4, t)
    out.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.5
        assert v == pytest.approx(1000 * 2 * 4 / 2.5)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_throughput(10, 1, 2, 4.0) == 5.0
