"""Work split and timing aggregation for several GPUs of one node.

Frames (and streams) are independent through the whole estimator -- every 2^n x 2^n
superblock is, since Haar windows never overlap (Eq. 1) -- so N GPUs run N replicas
that each take their own share of the frames; nothing is exchanged on the data path.
The only collective is on the host side of a measurement: the slowest replica's time
and the total of frames processed.
"""
from __future__ import annotations


def shard(n_units: int, rank: int, world: int) -> range:
    """Units (frames, streams) of this rank: round robin, disjoint, covering all."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return range(rank, n_units, world)


def aggregate(local_ms: float, local_units: int, device=None):
    """(max over ranks of local_ms, sum over ranks of local_units) with torch.distributed
    (gloo on CPU tensors, NCCL on CUDA tensors); the local values when not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms), int(local_units)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([int(local_units)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())
