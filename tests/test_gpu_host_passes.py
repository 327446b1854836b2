"""ktau_allpairs_host: passes over result sub-ranges with device-to-host copies overlapping the
next pass (Sec. 4.3.1) give exactly the device results, whatever the pass size."""
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


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("pass_pairs", [0, 1, 997, 10000, 10**9])
def test_host_passes_equal_device(ktau, path, pass_pairs):
    X = uniform_ties(300, 140, tie_frac=0.2, seed=path)
    Xd = torch.from_numpy(X).cuda()
    ref = ktau.allpairs(Xd, count_bits=32, options={"path": path})
    torch.cuda.synchronize()
    R = ref["ranked"]
    P = R.pairs
    lo, hi = 17, P - 5
    h = {"tau64": torch.full((hi - lo,), -9.0, dtype=torch.float64).pin_memory(),
         "tau32": torch.full((hi - lo,), -9.0, dtype=torch.float32).pin_memory(),
         "S": torch.full((hi - lo,), -9, dtype=torch.int32).pin_memory(),
         "n3": torch.full((hi - lo,), -9, dtype=torch.int32).pin_memory()}
    if pass_pairs == 1:
        lo, hi = 0, 4000  # one pair per pass would be too slow over the whole range
        h = {k: v[: hi - lo] for k, v in h.items()}
    ktau.ktau_allpairs_host(R, lo, hi, h["tau64"], h["tau32"], h["S"], h["n3"], 32,
                            {"path": path}, pass_pairs)
    for k in h:
        a = h[k].numpy()
        b = ref[k][lo:hi].cpu().numpy()
        assert np.array_equal(a.view(np.int64 if a.itemsize == 8 else np.int32),
                              b.view(np.int64 if b.itemsize == 8 else np.int32)), k
    R.free()


def test_host_passes_benchmark_size(ktau):
    X = gene_expression(16384, 128, seed=0)
    R = ktau.ktau_rank_prepare(torch.from_numpy(X).cuda())
    P = R.pairs
    t32 = torch.empty(P, dtype=torch.float32).pin_memory()
    S = torch.empty(P, dtype=torch.int32).pin_memory()
    ktau.ktau_allpairs_host(R, 0, P, None, t32, S, None, 32)
    Sd = torch.empty(P, dtype=torch.int32, device="cuda")
    ktau.ktau_allpairs(R, 0, P, None, None, Sd, None, 32)
    torch.cuda.synchronize()
    assert torch.equal(Sd.cpu(), S)
    assert torch.isfinite(t32).all() and t32.abs().max() <= 1.0
    R.free()


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_rank_prepare_from_host(ktau, dtype):
    """ktau_rank_prepare_host (host values, strided rows, pinned or pageable) gives the same ranked
    matrix as ktau_rank_prepare on the device copy, and rejects a NaN."""
    X = uniform_ties(70, 150, tie_frac=0.3, seed=9)
    if dtype == "i32":
        X = (X * 50).astype(np.int32)
    wide = np.zeros((70, 160), dtype=X.dtype)
    wide[:, :150] = X
    host = torch.from_numpy(wide)[:, :150]  # row stride 160
    for h in (host, host.pin_memory()):
        Rh = ktau.ktau_rank_prepare_host(h)
        Rd = ktau.ktau_rank_prepare(torch.from_numpy(X).cuda())
        for a, b in zip(ktau.ktau_ranked_export(Rh), ktau.ktau_ranked_export(Rd)):
            assert torch.equal(a, b)
        assert torch.equal(ktau.ktau_tie_counts(Rh), ktau.ktau_tie_counts(Rd))
        Rh.free()
        Rd.free()
    if dtype == "f32":
        bad = torch.from_numpy(X.copy())
        bad[3, 7] = float("nan")
        with pytest.raises(ktau.KtauError) as ei:
            ktau.ktau_rank_prepare_host(bad)
        assert ei.value.status == 2
