"""Error handling without a GPU fault: injected allocation failures surface as KTAU_ENOMEM and
leave the library usable; a bounded device wait that nothing satisfies gives up, raises the
status word (KTAU_ETIMEOUT through ktau_device_status) and the context keeps working; a pending
server request can be cancelled."""
import numpy as np
import pytest
import torch

from synthetic import gene_expression, uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def test_injected_allocation_failure(ktau):
    X = torch.from_numpy(uniform_ties(50, 77, seed=1)).cuda()
    ktau.ktau_debug_fail_alloc(0)
    try:
        with pytest.raises(ktau.KtauError) as ei:
            ktau.ktau_rank_prepare(X)
        assert ei.value.status == 4  # KTAU_ENOMEM
    finally:
        ktau.ktau_debug_fail_alloc(-1)
    # the first allocation (ranks) succeeds, the sign expansion fails
    ktau.ktau_debug_fail_alloc(1)
    try:
        R = ktau.ktau_rank_prepare(X)
        with pytest.raises(ktau.KtauError) as ei:
            ktau.ktau_prepare_signs(R)
        assert ei.value.status == 4
    finally:
        ktau.ktau_debug_fail_alloc(-1)
    R.free()
    res = ktau.allpairs(X)  # library still usable
    torch.cuda.synchronize()
    assert res["S"].numel() == 50 * 49 // 2


def test_bounded_wait_timeout_keeps_context(ktau):
    ktau.ktau_device_status()  # clear
    ktau.ktau_debug_wait_timeout(10_000_000)  # 10 ms
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_device_status()
    assert ei.value.status == 6  # KTAU_ETIMEOUT
    ktau.ktau_device_status()  # cleared
    X = torch.from_numpy(uniform_ties(40, 60, seed=2)).cuda()
    res = ktau.allpairs(X, options={"path": 2})  # tensor-core path still works
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    assert res["S"].numel() == 40 * 39 // 2


def test_server_cancellation(ktau):
    from paper_1704_03767_gb300.serving import QueryServer

    D = gene_expression(2048, 64, seed=3)
    srv = QueryServer(D, k=5, slots=1)
    big = [gene_expression(256, 64, seed=10 + i) for i in range(6)]
    reqs = [srv.submit(q) for q in big]
    cancelled = srv.cancel(reqs[-1])
    for r in reqs:
        r.done.wait()
    assert cancelled and reqs[-1].error == "cancelled" and reqs[-1].topk_idx is None
    assert all(r.error is None for r in reqs[:-1])
    srv.stop()
