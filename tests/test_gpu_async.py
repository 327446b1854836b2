"""Asynchronous rank preparation: the handle's statistics arrive behind an event and are read by
the first call that needs them. Results equal the synchronous form's (exact counts, tau against
the oracle), a NaN is reported by that first call, and handles that are never used or far
outnumber the pinned statistics slots are released and recycled."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_tau32, assert_tau64, oracle_full
from synthetic import uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


@pytest.mark.parametrize("path,shape", [(2, (300, 90)), (2, (520, 301)), (1, (70, 140))])
def test_async_matches_oracle(ktau, path, shape):
    m, n = shape
    X = uniform_ties(m, n, tie_frac=0.2, seed=m + n)
    Xd = torch.from_numpy(X).cuda()
    st = torch.cuda.current_stream()
    R = ktau.ktau_rank_prepare_async(Xd, st)
    if path == 2:
        ktau.ktau_prepare_signs(R, st)  # enqueued before the statistics are read
    P = m * (m - 1) // 2
    tau64 = torch.empty(P, dtype=torch.float64, device="cuda")
    tau32 = torch.empty(P, dtype=torch.float32, device="cuda")
    S = torch.empty(P, dtype=torch.int64, device="cuda")
    n3 = torch.empty(P, dtype=torch.int64, device="cuda")
    ktau.ktau_allpairs(R, 0, P, tau64, tau32, S, n3, 64, {"path": path}, st)
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    R.free()
    ref = oracle_full(X)
    assert np.array_equal(S.cpu().numpy(), ref["S"])
    assert np.array_equal(n3.cpu().numpy(), ref["n3"])
    assert_tau64(tau64.cpu().numpy(), ref["tau"])
    assert_tau32(tau32.cpu().numpy(), ref["tau"])


def test_async_nan_reported_on_first_use(ktau):
    X = np.random.default_rng(3).random((40, 30)).astype(np.float32)
    X[5, 11] = np.nan
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare_async(Xd)  # no error yet: the flag is still on its way
    P = 40 * 39 // 2
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    for _ in range(2):  # the first use and every later one
        with pytest.raises(ktau.KtauError) as ei:
            ktau.ktau_allpairs(R, 0, P, None, None, S, None, 32)
        assert ei.value.status == 2
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_allpairs_path(R)
    assert ei.value.status == 2
    R.free()


def test_async_handles_recycled(ktau):
    """More handles than pinned slots, most never used: each release returns its slot; a handle
    made while none is free takes the synchronous form."""
    X = uniform_ties(8, 20, seed=5)
    Xd = torch.from_numpy(X).cuda()
    live = [ktau.ktau_rank_prepare_async(Xd) for _ in range(4200)]
    torch.cuda.synchronize()
    P = 8 * 7 // 2
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    ref = oracle_full(X)["S"]
    for R in (live[0], live[-1]):
        ktau.ktau_allpairs(R, 0, P, None, None, S, None, 32, {"path": 1})
        torch.cuda.synchronize()
        assert np.array_equal(S.cpu().numpy().astype(np.int64), ref)
    for R in live:
        R.free_on(torch.cuda.current_stream())
    again = [ktau.ktau_rank_prepare_async(Xd) for _ in range(100)]
    for R in again:
        R.free()
