"""Sharding of an ensemble over processes (one GPU each).

The chains are independent (Sec. 3.1), so an ensemble splits into contiguous
global chain-id ranges with no exchange during the run; each shard passes its
range start to the library (`SlipSpring(..., chain_offset=...)`), so every
chain draws the same numbers as in an unsharded run.  Observables are FP64 sums
over chains, combined once at the end by a sum over shards.
"""
import numpy as np


def shard_range(total: int, world: int, rank: int):
    """(offset, count) of rank's contiguous share of `total` chains."""
    if not (0 <= rank < world) or total < world:
        raise ValueError("need 0 <= rank < world <= total")
    lo = rank * total // world
    hi = (rank + 1) * total // world
    return lo, hi - lo


def allreduce_sum(x, group=None):
    """Sum of a NumPy float64 array over the ranks of a torch.distributed group
    (returns x itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return np.asarray(x)
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()
