"""Replica sharding of independent right-hand sides over ranks.

The paper's production ran independent inversions spread over GPU nodes
(Acknowledgements: an 8-node Tesla cluster and NCSA Lincoln).  Every noise
vector or point source is independent, so ranks take disjoint contiguous index
ranges.  There is no data-path collective: each rank produces its own loops and
a host-side merge adds them in rank order, which makes the result identical
whatever the number of ranks.
"""

from __future__ import annotations

import numpy as np


def index_range(rank: int, world: int, total: int) -> tuple[int, int]:
    """Contiguous [first, first + count) share of `total` items for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad rank / world / total")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def merge_ordered(parts: list[np.ndarray]) -> np.ndarray:
    """Concatenate per-rank results (each indexed by its own items) in rank order."""
    return np.concatenate([np.asarray(p) for p in parts], axis=0)


def gather_to_root(local: np.ndarray, group=None) -> np.ndarray | None:
    """Gather every rank's array to rank 0 (torch.distributed, any backend) in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.ascontiguousarray(local))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.shape[0]], dtype=torch.int64), group=group)
    n_max = int(max(s.item() for s in sizes))
    pad = torch.zeros((n_max,) + tuple(t.shape[1:]), dtype=t.dtype)
    pad[: t.shape[0]] = t
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    if dist.get_rank(group) != 0:
        return None
    return merge_ordered([b[: int(s.item())].numpy() for b, s in zip(bufs, sizes)])
