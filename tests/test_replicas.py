"""The multi-GPU form of the benchmark runs replicas (single-source BFS does
not shard without a per-level exchange): the job's time is the slowest rank's,
its work the sum of all ranks'.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, edges = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, edges))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, edges in out:
        assert ms == 15.0 and edges == 3000.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_over_ranks(3.5, 42, 1, "cpu") == (3.5, 42.0)
