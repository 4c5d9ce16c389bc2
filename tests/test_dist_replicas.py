"""The benchmark's multi-rank path (one process per GPU, replicas, no collective on
the data path) on CPU: two gloo ranks, the barrier, the max over ranks of the timed
region, and the whole-job throughput of independent replicas."""
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


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, local, d = bench.dist_setup()
    assert (w, r) == (world, rank) and d is not None
    bench.barrier(d, torch)
    seconds = 2.0 + rank            # rank 1 is the slower replica
    t = bench.max_over_ranks(seconds, d, "cpu")
    rate = bench.replica_rate(10, seconds, d, "cpu")
    out.put((rank, t, rate))
    d.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 3.0                      # the max over ranks
        assert abs(rate - 2 * 10 / 3.0) < 1e-12   # 20 units over the slowest rank's 3 s
