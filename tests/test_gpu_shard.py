"""Sharded forms on one GPU (Sec. 4.4 static partition; every run here has one GPU): two processes
(gloo for the host-side gather) each compute their own contiguous range of the pair triangle
through the library's range argument, with no kernel waiting on the other process, and the
gathered result equals one call over the whole triangle; a query database split by rows into
shards, each shard's top-k merged on the host, equals the top-k over the whole database."""
import os
import socket

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_worker(rank, world, port, path, q):
    import torch.distributed as dist

    import paper_1704_03767_gb300 as k
    from paper_1704_03767_gb300.sharding import gather_slices, shard_range
    from synthetic import gene_expression

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    X = gene_expression(1500, 128, seed=7)  # the same matrix on every rank (replicated input)
    P = 1500 * 1499 // 2
    lo, hi = shard_range(P, world, rank)
    R = k.ktau_rank_prepare(torch.from_numpy(X).cuda())
    S = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
    t32 = torch.empty(hi - lo, dtype=torch.float32, device="cuda")
    k.ktau_allpairs(R, lo, hi, None, t32, S, None, 32, {"path": path})
    torch.cuda.synchronize()
    R.free()
    Sg = gather_slices(S.cpu(), world, P)
    tg = gather_slices(t32.cpu(), world, P)
    if rank == 0:
        q.put((Sg.numpy(), tg.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("path", [1, 2])
def test_two_rank_shards_equal_one_call(ktau, path):
    import torch.multiprocessing as mp

    from synthetic import gene_expression

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, path, q)) for r in range(2)]
    for p in procs:
        p.start()
    S, t32 = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    X = gene_expression(1500, 128, seed=7)
    ref = ktau.allpairs(torch.from_numpy(X).cuda(), count_bits=32, options={"path": path})
    torch.cuda.synchronize()
    assert np.array_equal(S, ref["S"].cpu().numpy())
    assert np.array_equal(t32.view(np.int32), ref["tau32"].cpu().numpy().view(np.int32))
    ref["ranked"].free()


def test_query_database_row_shards(ktau):
    from paper_1704_03767_gb300.sharding import merge_topk
    from synthetic import gene_expression

    n, k, b = 256, 100, 6
    D = gene_expression(5000, n, seed=3)
    Q = gene_expression(b, n, seed=4)
    Q[1] = D[4321]            # |tau| = 1 against row 4321
    D[2600] = D[1300]         # equal rows in different shards
    Qd = torch.from_numpy(Q).cuda()
    qh = ktau.ktau_rank_prepare(Qd)
    whole = ktau.ktau_rank_prepare(torch.from_numpy(D).cuda())
    idx = torch.empty((b, k), dtype=torch.int32, device="cuda")
    tk = torch.empty((b, k), dtype=torch.float64, device="cuda")
    Sw = torch.empty((b, 5000), dtype=torch.int32, device="cuda")
    ktau.ktau_query(whole, qh, None, Sw, None, 32, k, idx, tk)
    torch.cuda.synchronize()
    parts = []
    for lo, hi in ((0, 1700), (1700, 3400), (3400, 5000)):
        sh = ktau.ktau_rank_prepare(torch.from_numpy(np.ascontiguousarray(D[lo:hi])).cuda())
        m = hi - lo
        S = torch.empty((b, m), dtype=torch.int32, device="cuda")
        i_s = torch.empty((b, k), dtype=torch.int32, device="cuda")
        t_s = torch.empty((b, k), dtype=torch.float64, device="cuda")
        ktau.ktau_query(sh, qh, None, S, None, 32, k, i_s, t_s)
        T = ktau.ktau_tie_counts(sh)
        torch.cuda.synchronize()
        il = i_s.cpu().numpy().astype(np.int64)
        Sl, Tl = S.cpu().numpy(), T.cpu().numpy()
        parts.append({"offset": lo, "idx": il, "tau": t_s.cpu().numpy(),
                      "S": np.take_along_axis(Sl, il, axis=1), "T": Tl[il]})
        sh.free()
    gi, gt = merge_topk(parts, k, n)
    assert np.array_equal(gi, idx.cpu().numpy())
    assert np.array_equal(gt.view(np.int64), tk.cpu().numpy().view(np.int64))
    qh.free()
    whole.free()
