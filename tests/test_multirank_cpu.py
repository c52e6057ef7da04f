"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective), timing reduced as the maximum over ranks, whole-job throughput
summed over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)]      # each rank measured its own replica
    agg = bench.aggregate_max(times, dist, "cpu")
    value = bench.job_throughput(world, 1000.0, 10, agg[0])
    out.put((rank, agg, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, agg, value in res:
        assert agg == [2.0, 5.0, 0.5]                          # the slowest rank on every quantity
        assert value == pytest.approx(2 * 1000.0 * 10 / 2.0)   # both replicas' units over the max time


def test_single_rank_identity():
    import bench
    assert bench.aggregate_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_throughput(1, 8, 5, 2.0) == 20.0
