"""The channel-sharded frame on CPU: two gloo ranks each take their slice of
receive channels (a partial image: the oracle's image with the other
channels weighted 0) and the reduce-sum gives the whole frame's image; the
slicing rules."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    g = synth.Geometry(n_tx=8, n_ch=24, n_samples=256, out_dims=(9, 1, 11))
    g.out_min, g.out_max = (-1e-3, 0.0, 2e-3), (1e-3, 0.0, 4e-3)
    r = np.random.default_rng(3).normal(size=(8, 24, 256))
    return g, r


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2512_11086_gb300 import shard
    g, r = _case()
    off, cnt = shard.channel_slices(g.n_ch, world)[rank]
    w = np.zeros(g.n_ch)
    w[off:off + cnt] = 1.0
    part = torch.from_numpy(oracle.das(g, r, w=w))
    shard.reduce_image(part)
    out[rank] = part.numpy().tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_channel_shards_sum_to_the_frame():
    import oracle
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
    g, r = _case()
    want = oracle.das(g, r)
    for rank in range(2):
        np.testing.assert_allclose(np.array(out[rank]), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_channel_slices():
    from paper_2512_11086_gb300 import shard
    assert shard.channel_slices(128, 4) == [(0, 32), (32, 32), (64, 32), (96, 32)]
    assert shard.channel_slices(40, 3) == [(0, 16), (16, 16), (32, 8)]
    with pytest.raises(ValueError):
        shard.channel_slices(12, 2)
    with pytest.raises(ValueError):
        shard.channel_slices(16, 3)
