"""Channel-sharded beamforming of one frame over several GPUs (one process per
GPU): rank r beamforms its slice of receive channels with a plan whose
channels are that slice of the whole array (rcbf_params.rx_channel_offset /
rx_channels_total), and the partial images add in one reduce-sum over
torch.distributed, the only exchange the sharded frame needs (Eq. (1) is a
sum over channels). Frames, by contrast, shard with no collective at all.
"""
from __future__ import annotations

from typing import List, Tuple

from . import make_params


def channel_slices(n_ch: int, world: int, multiple: int = 8) -> List[Tuple[int, int]]:
    """(offset, count) of each rank's channels: contiguous, in rank order,
    counts multiples of `multiple` (the tiled DAS's channel chunk) as evenly
    as possible."""
    if world < 1 or n_ch % multiple or n_ch // multiple < world:
        raise ValueError("n_ch must be a multiple of %d with at least one chunk per rank" % multiple)
    chunks = n_ch // multiple
    base, extra = divmod(chunks, world)
    out, off = [], 0
    for r in range(world):
        cnt = (base + (1 if r < extra else 0)) * multiple
        out.append((off, cnt))
        off += cnt
    return out


def shard_params(g, rank: int, world: int, **kw):
    """rcbf_params of rank `rank`'s channel slice of geometry g (the other
    fields as make_params gives them)."""
    off, cnt = channel_slices(int(g.n_ch), world)[rank]
    p = make_params(g, **kw)
    p.n_ch = cnt
    p.rx_channel_offset = off
    p.rx_channels_total = int(g.n_ch)
    return p


def reduce_image(image, group=None):
    """Sum the ranks' partial images in place (all ranks end with the image)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(image, op=dist.ReduceOp.SUM, group=group)
    return image
