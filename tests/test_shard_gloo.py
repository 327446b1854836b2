"""Multi-process logic on CPU (gloo, world size 2): every rank computes its static shard of the
pair range (Sec. 4.4) -- here with the CPU oracle, since the box has no GPU -- and the gathered
shards equal the single-process result; the max-over-ranks timing reduction is checked too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1704_03767_gb300.sharding import gather_slices, max_over_ranks, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_q):
    import oracle
    from synthetic import uniform_ties

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = uniform_ties(37, 50, seed=11)
    P = 37 * 36 // 2
    lo, hi = shard_range(P, world, rank)
    part = oracle.allpairs(X, method="knight", p_begin=lo, p_end=hi)
    S = gather_slices(torch.from_numpy(part["S"]), world, P)
    tau = gather_slices(torch.from_numpy(part["tau"]), world, P)
    t = max_over_ranks(1.0 + rank)
    if rank == 0:
        out_q.put((S.numpy(), tau.numpy(), t))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_disjointly():
    for total in (0, 1, 7, 2016, 134209536):
        for world in (1, 2, 3, 8):
            rs = [shard_range(total, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))


def test_two_rank_gather_matches_single_process():
    import oracle
    from synthetic import uniform_ties

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    S, tau, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.allpairs(uniform_ties(37, 50, seed=11), method="knight")
    assert np.array_equal(S, ref["S"])
    assert np.array_equal(tau, ref["tau"], equal_nan=True)
    assert t == 2.0


def test_merge_topk_of_row_shards_equals_whole_database():
    """Query search with the database split by rows (Sec. 4.4 partition): each shard's exact top-k
    (oracle order) merged on the host equals the top-k over the whole database, including rows
    tied in |tau| across shards, a constant row (NaN, last) and a constant query."""
    import oracle
    from paper_1704_03767_gb300.sharding import merge_topk

    g = np.random.default_rng(5)
    n = 12
    D = g.integers(0, 5, (23, n)).astype(float)
    D[15] = D[2]      # equal |tau| to row 2, in another shard
    D[20] = -D[2]
    D[9] = 3.0        # constant row
    Q = g.integers(0, 6, (3, n)).astype(float)
    Q[2] = 1.0        # constant query
    k = 7
    ref = oracle.query_topk(Q, D, k)
    n0 = n * (n - 1) // 2
    parts = []
    for lo, hi in ((0, 8), (8, 16), (16, 23)):
        r = oracle.rect(Q, D[lo:hi])
        Du = [n0 - int(r["n1"][i, 0]) for i in range(3)]
        kk = min(k, hi - lo)
        idx = [oracle.topk_order(r["S"][i], Du[i], n0 - r["n2"][i], kk) for i in range(3)]
        parts.append({"offset": lo, "idx": idx,
                      "tau": [r["tau"][i, idx[i]] for i in range(3)],
                      "S": [r["S"][i, idx[i]] for i in range(3)],
                      "T": [r["n2"][i, idx[i]] for i in range(3)]})
    idx, tau = merge_topk(parts, k, n)
    assert np.array_equal(idx, ref["topk_idx"])
    assert np.array_equal(np.isnan(tau), np.isnan(ref["topk_tau"]))
    assert np.array_equal(np.nan_to_num(tau), np.nan_to_num(ref["topk_tau"]))
