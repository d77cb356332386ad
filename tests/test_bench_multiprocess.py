"""bench.py's multi-rank bookkeeping on CPU: two gloo ranks, each with its own
frames, report the slowest rank's time and the units of the whole job."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(3.5, 7.0) == (3.5, 7.0)
