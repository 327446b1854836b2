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
