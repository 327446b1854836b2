"""Static partition of the pair range over p processes (Sec. 4.4: process i takes ids
[i*ceil(P/p), (i+1)*ceil(P/p))), and the host-side pieces of running one shard per GPU: the
shard's range for ktau_allpairs, the gather of the disjoint output slices, the max-over-ranks
timing used by the benchmark, and the exact merge of per-shard top-k candidates when a query
database is split by rows. The shards never exchange data while computing."""
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


def merge_topk(parts, k: int, n: int):
    """Exact top-k of a query batch over a database split by rows across shards (Sec. 4.4's
    static partition applied to the query search): each shard's own top-k candidates are merged
    on the host in the library's order -- |tau| descending by the exact rational S^2 / D_v (D_u is
    common to a query row), equal values by the smaller global row index, NaN last.

    parts: one dict per shard with "offset" (its first global row), "idx" [b][k_s] (shard-local
    rows), "tau" [b][k_s], "S" [b][k_s] and "T" [b][k_s] (the tie counts of those database rows).
    Returns (idx [b][k] global rows, tau [b][k]) as numpy arrays."""
    import numpy as np

    n0 = n * (n - 1) // 2
    b = len(parts[0]["idx"])
    idx = np.zeros((b, k), np.int64)
    tau = np.zeros((b, k), np.float64)
    for q in range(b):
        cand = []
        for p in parts:
            for j, t, s, tv in zip(p["idx"][q], p["tau"][q], p["S"][q], p["T"][q]):
                g = int(p["offset"]) + int(j)
                dv = n0 - int(tv)
                if np.isnan(t) or dv == 0:
                    cand.append(((1, 0, 1), g, float(t)))
                else:  # compare S^2 / D_v exactly: the key (0, -S^2, D_v) ordered by cross products
                    cand.append(((0, int(s) * int(s), dv), g, float(t)))

        def key(c):
            (nan, s2, dv), g, _ = c
            return (nan, _Frac(-s2, dv), g)

        cand.sort(key=key)
        for i, (_, g, t) in enumerate(cand[:k]):
            idx[q, i] = g
            tau[q, i] = t
    return idx, tau


def _Frac(num, den):
    from fractions import Fraction

    return Fraction(num, den)
