"""The multi-rank host logic of bench.py on CPU with gloo, world size 2: each
rank runs an independent replica (no collective on the data path); the job's
time is the slowest rank's, and the throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup()
    my_seconds = 1.0 + rank  # rank 1 is the slow one
    slowest = bench.reduce_max(my_seconds, dist, "cpu")
    value = bench.whole_job_throughput(1000.0, ws, slowest)
    out.put((r, ws, local, slowest, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
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
    for r, (rank, ws, local, slowest, value) in enumerate(res):
        assert rank == r and local == r and ws == 2
        assert slowest == 2.0  # max over ranks
        assert value == 2 * 1000.0 / 2.0  # all ranks' units over the slowest time
