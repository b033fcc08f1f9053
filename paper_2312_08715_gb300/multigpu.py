"""Host-side plumbing for running the path on several GPUs (one process per GPU).

Hypotheses and scenes are independent, so the path shards without any data exchange: each
rank renders and scores its own contiguous range of hypotheses (or its own scenes). The one
step that spans ranks when a single coarse-to-fine stage is split over GPUs is the log
normaliser of the categorical over cells (Sec. III-B): each rank's b3d_lse_resample gives
its local log Z_r, and the global log Z is the log-sum-exp of those few numbers, gathered
with one all-gather. Timings are combined by their maximum over ranks.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """Contiguous [begin, end) of n hypotheses owned by rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def combine_logz(local_logz, group=None):
    """Global log normaliser from each rank's local one (a 1-element tensor); ranks with no
    hypotheses pass -inf."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local_logz) for _ in range(world)]
    dist.all_gather(parts, local_logz, group=group)
    return torch.logsumexp(torch.cat(parts).double(), dim=0)


def max_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
