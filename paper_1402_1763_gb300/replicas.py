"""Independent chains across processes (Sec. 3.4: chains need no communication).

Each rank runs its own context with its own chain ids; the only cross-rank
traffic is host-side bookkeeping: a barrier around timed regions and the
maximum of the ranks' elapsed times.  No collective touches the data path.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world_size, local_rank) from the torchrun environment, else (0, 1, 0)."""
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def chain_id_base(rank: int, chains_per_rank: int) -> int:
    """First chain id of a rank: ranks draw disjoint Philox streams."""
    return rank * chains_per_rank


def max_over_ranks(value: float, dist=None) -> float:
    """Max of a host float over all ranks (identity for a single process)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist=None):
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
