"""One search split over the ranks of a process group.

Rank g of G owns the start positions [g S / G, (g + 1) S / G) of the
S = n - m + 1 starts of a pattern of length m in a text of n bytes, and
needs the text bytes from its first start to m - 1 past its last one (the
halo). Every start is tested by exactly one rank (Algorithm 1 tests each
start independently), so the counts add up: one all-reduce gives the total.
A report is the concatenation of the ranks' ascending position lists in
rank order: an all-gather of the counts gives each rank its first rank in
the output.

The local search is passed in (on a GPU rank: sm_count / sm_report on the
rank's slice of a device-resident text); this module holds only the split
and the exchange, over torch.distributed (NCCL for GPU ranks, gloo on CPU).
"""
from __future__ import annotations


def start_range(n: int, m: int, rank: int, world: int) -> tuple[int, int]:
    """The starts [s0, s1) that rank `rank` of `world` owns (empty when m > n)."""
    starts = max(n - m + 1, 0) if m >= 1 else 0
    return starts * rank // world, starts * (rank + 1) // world


def text_range(n: int, m: int, rank: int, world: int) -> tuple[int, int]:
    """The text bytes [b0, b1) the rank reads: its starts plus the (m - 1)-byte halo."""
    s0, s1 = start_range(n, m, rank, world)
    if s1 <= s0:
        return s0, s0
    return s0, min(s1 + m - 1, n)


def sharded_count(local_count, n: int, m: int, group=None) -> int:
    """Total count over the group. local_count(b0, b1) returns the number of
    matches that start in text bytes [b0, b1) and end inside them."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    b0, b1 = text_range(n, m, rank, world)
    c = int(local_count(b0, b1)) if b1 - b0 >= m else 0
    t = torch.tensor([c], dtype=torch.int64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


def sharded_report(local_report, n: int, m: int, group=None):
    """(first, positions, total): this rank's ascending positions (absolute in
    the text) and their first rank in the group's output, and the total
    count. local_report(b0, b1) returns the positions relative to b0 of the
    matches inside text bytes [b0, b1), ascending."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    b0, b1 = text_range(n, m, rank, world)
    pos = local_report(b0, b1) if b1 - b0 >= m else []
    mine = torch.tensor([len(pos)], dtype=torch.int64, device=_device(group))
    counts = [torch.zeros(1, dtype=torch.int64, device=mine.device) for _ in range(world)]
    dist.all_gather(counts, mine, group=group)
    counts = [int(c.item()) for c in counts]
    return sum(counts[:rank]), [b0 + int(p) for p in pos], sum(counts)


def _device(group):
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")
