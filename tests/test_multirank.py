"""Host logic of the N > 1 bench path (independent replicas): max-over-ranks
timing and whole-job throughput, run as two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank        # rank 1 is the slowest
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (t, bench.job_throughput(world, 4, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t, v = out[r]
        assert t == 150.0                  # every rank reports the slowest rank's time
        assert abs(v - 2 * 4 / 0.150) < 1e-9   # solves of all ranks / slowest time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(1, 10, 500.0) == 20.0
