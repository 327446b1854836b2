"""Static partition of the pair range over p processes (Sec. 4.4: process i takes ids
[i*ceil(P/p), (i+1)*ceil(P/p))), and the host-side pieces of running one shard per GPU: the
shard's range for ktau_allpairs, the gather of the disjoint output slices, and the
max-over-ranks timing used by the benchmark. The shards never exchange data while computing."""
from __future__ import annotations


def shard_range(total: int, world: int, rank: int):
    """[lo, hi) of rank `rank` among `world` equal contiguous ranges of [0, total)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    per = -(-total // world)
    lo = min(total, rank * per)
    hi = min(total, (rank + 1) * per)
    return lo, hi


def gather_slices(local, world: int, total: int, group=None):
    """All ranks' disjoint slices (1-D torch tensors, in rank order) concatenated on every rank.
    Slices may differ in length by the last-rank remainder, so they are padded for all_gather."""
    import torch
    import torch.distributed as dist

    per = -(-total // world)
    buf = torch.zeros(per, dtype=local.dtype, device=local.device)
    buf[: local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = []
    for r, p in enumerate(parts):
        lo, hi = shard_range(total, world, r)
        out.append(p[: hi - lo])
    return torch.cat(out)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest `value` over all ranks (the benchmark's whole-job time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
