"""Host-side partition and gather of a rollout split over ranks.

The (particle, sequence) simulations of a rollout are independent (Sec. 2.2),
so a rollout can be split by sequences, by particles or both, each shard run
with voila_rollout_shard, whose noise counters are those of the whole problem.
This module holds the host logic only: which block a rank owns and how the
shards' returns are put back together, in a fixed order so that the result
does not depend on timing.

  split by sequences: J of the whole problem = the shards' J side by side,
    in rank order (bit-identical to the unsharded call);
  split by particles: J = the shards' partial sums added in rank order
    (equal to the unsharded J up to the order of the FP64 additions).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch


def shard_range(total: int, world: int, rank: int) -> Tuple[int, int]:
    """(offset, count) of rank's contiguous block of `total` items; the first
    total % world ranks hold one item more."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard geometry")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def combine_sequence_shards(parts: Sequence[torch.Tensor]) -> torch.Tensor:
    """J of a sequence-split rollout from the shards' J, in rank order."""
    return torch.cat(list(parts))


def combine_particle_shards(parts: Sequence[torch.Tensor]) -> torch.Tensor:
    """J of a particle-split rollout: the shards' partial sums added in rank order."""
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def _all_gather_padded(part: torch.Tensor, counts: List[int], group=None) -> List[torch.Tensor]:
    import torch.distributed as dist
    world = dist.get_world_size(group)
    width = max(counts)
    buf = torch.zeros(width, dtype=part.dtype, device=part.device)
    buf[: part.numel()] = part
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    return [b[:c] for b, c in zip(bufs, counts)]


def gather_sequence_shards(part: torch.Tensor, K_total: int, group=None) -> torch.Tensor:
    """Every rank's J of a sequence-split rollout (rank r holds shard_range(K_total,
    world, r)), gathered and concatenated in rank order on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    counts = [shard_range(K_total, world, r)[1] for r in range(world)]
    return combine_sequence_shards(_all_gather_padded(part, counts, group))


def reduce_particle_shards(part: torch.Tensor, group=None) -> torch.Tensor:
    """J of a particle-split rollout on every rank: the ranks' partial sums
    gathered and added in rank order (not an all-reduce, whose summation order
    is the library's choice)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    return combine_particle_shards(_all_gather_padded(part, [part.numel()] * world, group))
