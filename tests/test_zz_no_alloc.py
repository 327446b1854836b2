"""ktau_allpairs_noalloc against ktau_allpairs on the same inputs, through the C ABI.

The entry point serves callers that cannot allocate device memory where they need the result (a
plug-in inside a host framework's memory budget, a real-time loop that may not call cudaMalloc or
cudaFree). The tests call it twice in a row: the fixed scratch array keeps the previous call's
contents, so the second call also checks that nothing stale leaks into it. While it runs, the
library's allocation hook is set to fail every allocation, and the device's free memory is
compared before and after, so an allocation inside the call would fail the test.
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


@pytest.fixture(scope="module", autouse=True)
def warm(ktau):
    """First calls on the device: the array's address is looked up and CUDA loads the kernels'
    modules (lazy loading reserves device memory for code and globals then), so the free-memory
    checks below start from a loaded library. Short and long rows reach every kernel used."""
    for m, n in ((3, 40), (3, 1100)):
        Xd = torch.rand((m, n), device="cuda")
        o = _outs(3, 64)
        ktau.ktau_allpairs_noalloc(Xd, 0, 3, o["tau64"], o["tau32"], o["S"], o["n3"], 64)
        o = _outs(3, 32)
        ktau.ktau_allpairs_noalloc(Xd, 0, 3, o["tau64"], o["tau32"], o["S"], o["n3"], 32)
    torch.cuda.synchronize()


def _noalloc_call(ktau, Xd, P, o, count_bits):
    """One call with every library allocation made to fail and device memory watched."""
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ktau.ktau_debug_fail_alloc(0)
    try:
        ktau.ktau_allpairs_noalloc(Xd, 0, P, o["tau64"], o["tau32"], o["S"], o["n3"], count_bits)
        torch.cuda.synchronize()
    finally:
        ktau.ktau_debug_fail_alloc(-1)
    assert torch.cuda.mem_get_info()[0] == free0


def _compare(ktau, X, count_bits):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    m = X.shape[0]
    P = m * (m - 1) // 2
    o = _outs(P, count_bits)
    _noalloc_call(ktau, Xd, P, o, count_bits)
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


def test_noalloc_long_vectors_twice(ktau):
    """n > 1024: the CTA-per-variable rank kernel and the CTA-per-pair merge mapping."""
    X = uniform_ties(150, 1500, seed=4)
    _compare(ktau, X, 32)
    _compare(ktau, X[::-1].copy(), 64)


def test_noalloc_rejects_oversized_input(ktau):
    X = torch.rand((40000, 128), device="cuda")
    S = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_allpairs_noalloc(X, 0, 1, None, None, S, None, 32)
    assert ei.value.status == 3 and "scratch" in ei.value.message
