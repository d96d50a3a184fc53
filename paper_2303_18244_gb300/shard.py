"""Event sharding across ranks (one process per GPU).

Events are independent (paper Sect. 1: one matrix element per event, no
communication between events), so a multi-GPU run gives each rank its own
contiguous block of events and needs no collective on the data path: weak
scaling.  The only collectives are host-side bookkeeping around the timed
region: a barrier on both sides and the maximum of the ranks' times.
"""
from __future__ import annotations


def event_block(rank: int, world: int, nevt_per_rank: int) -> tuple[int, int]:
    """(first event index, count) of a rank's block of the global event stream."""
    if not (0 <= rank < world) or nevt_per_rank < 0:
        raise ValueError("bad rank/world/nevt")
    return rank * nevt_per_rank, nevt_per_rank


def max_over_ranks(values, device=None):
    """Element-wise maximum over ranks of a list of floats (identity when not
    distributed).  Uses the default process group (gloo on CPU, nccl on GPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
