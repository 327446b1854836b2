"""Kernel trace: every library launch is recorded in launch order with a positive CUDA-event time,
and the name filter restricts the records to one kernel without changing the results."""
import numpy as np
import pytest
import torch

from gpu_helpers import oracle_full
from synthetic import uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _step(ktau, Xd, P, S, n3):
    st = torch.cuda.current_stream()
    R = ktau.ktau_rank_prepare_async(Xd, st)
    ktau.ktau_prepare_signs(R, st)
    ktau.ktau_allpairs(R, 0, P, None, None, S, n3, 32, {"path": 2}, st)
    torch.cuda.synchronize()
    R.free()


def test_trace_all_and_filtered(ktau):
    X = uniform_ties(4100, 40, tie_frac=0.1, seed=9)  # m >= 4096: tie lists on the side stream
    m = X.shape[0]
    P = m * (m - 1) // 2
    Xd = torch.from_numpy(X).cuda()
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    n3 = torch.empty(P, dtype=torch.int32, device="cuda")
    ktau.ktau_trace_collect()
    try:
        ktau.ktau_trace_filter(None)
        ktau.ktau_trace_enable(True)
        _step(ktau, Xd, P, S, n3)
        full = ktau.ktau_trace_collect()
        names = [k for k, _ in full]
        for k in ("rank_kernel", "sign_expand_kernel", "contract_kernel"):
            assert k in names
        assert names.index("rank_kernel") < names.index("sign_expand_kernel") < \
            names.index("contract_kernel")
        assert all(t > 0 for _, t in full)
        ktau.ktau_trace_filter("contract_kernel")
        _step(ktau, Xd, P, S, n3)
        only = ktau.ktau_trace_collect()
        assert [k for k, _ in only] == ["contract_kernel"] and only[0][1] > 0
    finally:
        ktau.ktau_trace_enable(False)
        ktau.ktau_trace_filter(None)
        ktau.ktau_trace_collect()
    ref = oracle_full(X[:300])  # first 300 rows: their pairs lead the packed triangle per row
    Sh = S.cpu().numpy().astype(np.int64)
    # row i's pairs start at i(2m - i - 1)/2; compare pairs among the first rows
    for i in range(0, 299, 37):
        base = i * (2 * m - i - 1) // 2
        rbase = i * (2 * 300 - i - 1) // 2
        assert np.array_equal(Sh[base:base + (299 - i)], ref["S"][rbase:rbase + (299 - i)])
