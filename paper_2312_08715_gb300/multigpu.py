"""Host-side plumbing for running the path on several GPUs (one process per GPU).

Hypotheses and scenes are independent, so the path shards without any data exchange: each
rank renders and scores its own contiguous range of hypotheses (or its own scenes). The one
step that spans ranks when a single coarse-to-fine stage is split over GPUs is the
categorical over cells (Sec. III-B): its normaliser and its draws.
  1. Each rank forms its shard's log normaliser log Z_r (b3d_lse_resample with no draws).
  2. One all-gather of those numbers gives log Z = logsumexp_r log Z_r and each rank's share
     of the probability, mass_r = exp(log Z_r - log Z), and the share of the ranks before it.
  3. Each rank draws with b3d_lse_resample_shard: draw k (a counter-based uniform u_k every
     rank can form) belongs to the rank whose interval [before_r, before_r + mass_r) holds
     u_k, which finds its index inside its shard; other ranks write -1.
  4. One all-reduce (maximum) of the draw vectors gives every rank every draw.
In exact arithmetic the draws are those of the unsplit vector. Timings are combined by
their maximum over ranks.
"""
from __future__ import annotations

import math


def shard_range(n: int, rank: int, world: int):
    """Contiguous [begin, end) of n hypotheses owned by rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard_masses(logz_all, rank: int):
    """From every rank's shard log normaliser (-inf for an empty shard): the global log Z,
    the probability mass of the ranks before ``rank`` and ``rank``'s own mass. The last rank's
    mass runs to 1, so that every uniform in [0, 1) has an owner despite rounding."""
    finite = [z for z in logz_all if z > -math.inf]
    if not finite:
        return -math.inf, 0.0, 0.0
    top = max(finite)
    logz = top + math.log(sum(math.exp(z - top) for z in finite))
    masses = [math.exp(z - logz) if z > -math.inf else 0.0 for z in logz_all]
    before = min(1.0, sum(masses[:rank]))
    mass = 1.0 - before if rank == len(logz_all) - 1 else min(masses[rank], 1.0 - before)
    return logz, before, mass


def combine_logz(local_logz, group=None):
    """Global log normaliser from each rank's local one (a 1-element tensor); ranks with no
    hypotheses pass -inf."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local_logz) for _ in range(world)]
    dist.all_gather(parts, local_logz, group=group)
    return torch.logsumexp(torch.cat(parts).double(), dim=0)


def gather_logz(local_logz: float, group=None):
    """Every rank's shard log normaliser, on every rank (one all-gather of 8-byte values)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.tensor([float(local_logz)], dtype=torch.float64)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return [float(p.item()) for p in parts]


def gather_draws(idx, logq, group=None):
    """Combine the ranks' draw vectors (-1 / -inf where another rank owns a draw) into the
    full vectors on every rank: one all-reduce (maximum) of each. Tensors are updated in
    place and returned; they must live where the process group's backend works (host
    tensors for gloo, device tensors for nccl)."""
    import torch.distributed as dist
    dist.all_reduce(idx, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(logq, op=dist.ReduceOp.MAX, group=group)
    return idx, logq


def sharded_resample(ctx, ll_local, index_base: int, m: int, seed: int, stage: int, group=None):
    """Draws of the categorical over the whole split score vector, on every rank: this rank's
    scores ``ll_local`` (a device tensor) are [index_base, index_base + n) of it. Returns
    (log Z, idx [m] int32, logq [m]) as device tensors; every rank gets the same draws."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    z_local, _, _ = ctx.lse_resample(ll_local, 0, seed, stage)
    logz_all = gather_logz(float(z_local.item()), group)
    logz, before, mass = shard_masses(logz_all, rank)
    _, idx, logq = ctx.lse_resample_shard(ll_local, m, seed, stage, before, mass, logz, index_base)
    on_host = dist.get_backend(group) == "gloo"
    i = idx.to(torch.int64).cpu() if on_host else idx.to(torch.int64)
    q = logq.cpu() if on_host else logq
    gather_draws(i, q, group)
    return logz, i.to(device=idx.device, dtype=torch.int32), q.to(idx.device)


def max_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
