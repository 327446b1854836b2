"""Continuous-batching server: batches that arrive while others run are admitted as slots and
memory free up, overlap on the device, and each batch's result is identical to running it
alone (and to the oracle's exact top-k)."""
import numpy as np
import pytest
import torch

import oracle
from synthetic import gene_expression, query_batch_sizes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def test_results_alone_equal_results_in_the_mix(ktau):
    from paper_1704_03767_gb300.serving import QueryServer

    D = gene_expression(4096, 256, seed=0)
    sizes = query_batch_sizes(24, max_batch=64, seed=5)
    batches = [gene_expression(b, 256, seed=100 + i) for i, b in enumerate(sizes)]
    # alone: one slot, one batch at a time
    alone = QueryServer(D, k=25, slots=1)
    ref = []
    for q in batches:
        r = alone.submit(q)
        r.done.wait()
        assert r.error is None, r.error
        ref.append((r.topk_idx.copy(), r.topk_tau.copy()))
    alone.stop()
    # in the mix: 4 slots, everything submitted at once; pending batches are merged into
    # shared launches (rows of several requests in one contraction) ...
    mix = QueryServer(D, k=25, slots=4)
    reqs = [mix.submit(q) for q in batches]
    for r in reqs:
        r.done.wait()
        assert r.error is None, r.error
    for r, (ri, rt) in zip(reqs, ref):
        assert np.array_equal(r.topk_idx, ri)
        assert np.array_equal(r.topk_tau.view(np.int64), rt.view(np.int64))
    launches = {}
    for rid, slot, adm, fin in mix.timeline:
        launches.setdefault((slot, adm), []).append(rid)
    assert max(len(v) for v in launches.values()) > 1  # some launch served several requests
    mix.stop()
    # ... and without merging, batches run concurrently on different slots.
    sep = QueryServer(D, k=25, slots=4, merge=False)
    reqs2 = [sep.submit(q) for q in batches]
    for r, (ri, rt) in zip(reqs2, ref):
        r.done.wait()
        assert r.error is None, r.error
        assert np.array_equal(r.topk_idx, ri)
        assert np.array_equal(r.topk_tau.view(np.int64), rt.view(np.int64))
    tl = sorted(sep.timeline, key=lambda t: t[2])
    overlaps = sum(1 for a, b in zip(tl, tl[1:]) if b[2] < a[3] and b[1] != a[1])
    assert overlaps > 0
    sep.stop()
    # exact top-k against the oracle for one small batch
    i = int(np.argmin(sizes))
    o = oracle.query_topk(batches[i], D, 25)
    assert np.array_equal(reqs[i].topk_idx, o["topk_idx"])


def test_memory_admission_serialises(ktau):
    from paper_1704_03767_gb300.serving import QueryServer

    D = gene_expression(2048, 128, seed=1)
    probe = QueryServer(D, k=10, slots=4)
    need = probe.footprint(32)
    probe.stop()
    srv = QueryServer(D, k=10, slots=4, mem_budget=int(need * 1.5))  # one batch at a time
    reqs = [srv.submit(gene_expression(32, 128, seed=50 + i)) for i in range(6)]
    for r in reqs:
        r.done.wait()
        assert r.error is None
    tl = sorted(srv.timeline, key=lambda t: t[2])
    assert all(b[2] >= a[3] for a, b in zip(tl, tl[1:]))  # never two in flight
    big = srv.submit(gene_expression(512, 128, seed=9))    # larger than the whole budget
    big.done.wait()
    assert big.error is not None and "budget" in big.error
    srv.stop()
