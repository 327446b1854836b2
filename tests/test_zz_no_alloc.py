"""ktau_allpairs_noalloc (the entry point for callers that cannot allocate device memory) against
ktau_allpairs on the same inputs, twice in a row through the C ABI: the fixed scratch array keeps
the previous call's contents, so the second call also checks that nothing stale leaks into it.
Collected last on purpose (file name), so a failure here cannot hide other failures."""
import numpy as np
import pytest
import torch

from synthetic import gene_expression, uniform_ties

pytestmark = pytest.mark.gpu

TAU_RTOL = 1e-12


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _outs(P, count_bits):
    cdt = torch.int32 if count_bits == 32 else torch.int64
    return {"tau64": torch.full((P,), 3.0, dtype=torch.float64, device="cuda"),
            "tau32": torch.full((P,), 3.0, dtype=torch.float32, device="cuda"),
            "S": torch.full((P,), -1, dtype=cdt, device="cuda"),
            "n3": torch.full((P,), -1, dtype=cdt, device="cuda")}


def _compare(ktau, X, count_bits):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    m = X.shape[0]
    P = m * (m - 1) // 2
    o = _outs(P, count_bits)
    ktau.ktau_allpairs_noalloc(Xd, 0, P, o["tau64"], o["tau32"], o["S"], o["n3"], count_bits)
    ref = ktau.allpairs(Xd, count_bits=count_bits, options={"path": ktau.KTAU_PATH_MERGE})
    torch.cuda.synchronize()
    assert torch.equal(o["S"], ref["S"])
    assert torch.equal(o["n3"], ref["n3"])
    a, b = o["tau64"].cpu().numpy(), ref["tau64"].cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b)
    assert (np.abs(a[ok] - b[ok]) <= TAU_RTOL * np.abs(b[ok])).all()
    a, b = o["tau32"].cpu().numpy(), ref["tau32"].cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[~np.isnan(b)], b[~np.isnan(b)])
    ref["ranked"].free()


def test_noalloc_matches_allpairs_twice(ktau):
    X1 = uniform_ties(64, 200, seed=0)
    X1[5] = 0.25  # constant variable
    X2 = gene_expression(1000, 128, seed=3)
    _compare(ktau, X1, 64)
    _compare(ktau, X2, 32)  # second call reuses the scratch left by the first


def test_noalloc_rejects_oversized_input(ktau):
    X = torch.rand((40000, 128), device="cuda")
    S = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_allpairs_noalloc(X, 0, 1, None, None, S, None, 32)
    assert ei.value.status == 3 and "scratch" in ei.value.message
