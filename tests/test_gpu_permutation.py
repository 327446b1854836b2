"""Permutation test of every pair on the GPU (ktau_permutation_exceed) against the oracle:
exceedance counts bit-exact, for FP8 and FP4 operands, pair sub-ranges, identity relabellings and
the p-value convenience."""
import numpy as np
import pytest
import torch

import oracle
from synthetic import permutations, uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _exceed(ktau, X, perms, p_begin=0, p_end=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    if p_end is None:
        p_end = R.pairs
    S = torch.empty(p_end - p_begin, dtype=torch.int32, device="cuda")
    ktau.ktau_allpairs(R, p_begin, p_end, None, None, S, None, 32)
    exc = torch.zeros(p_end - p_begin, dtype=torch.uint32, device="cuda")
    ktau.ktau_permutation_exceed(R, torch.from_numpy(perms).cuda(), S, exc, p_begin, p_end)
    torch.cuda.synchronize()
    R.free()
    return exc.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("m,n,B", [(70, 50, 6), (300, 120, 3), (40, 300, 3)])
def test_matches_oracle(ktau, m, n, B):
    X = uniform_ties(m, n, tie_frac=0.3, seed=m + n)
    X[5] = X[6]  # a duplicated variable (|S| at its maximum)
    X[7] = 1.0   # a constant variable (S = 0 for every relabelling)
    perms = permutations(B, n, seed=m)
    got = _exceed(ktau, X, perms)
    ref = oracle.permutation_exceed(X, perms)
    assert np.array_equal(got, ref)


def test_ranges_and_identity(ktau):
    X = uniform_ties(90, 64, tie_frac=0.2, seed=21)
    perms = permutations(4, 64, seed=22)
    P = 90 * 89 // 2
    full = _exceed(ktau, X, perms)
    lo, hi = 1000, 2500
    assert np.array_equal(_exceed(ktau, X, perms, lo, hi), full[lo:hi])
    ident = np.tile(np.arange(64, dtype=np.uint16), (3, 1))
    assert np.all(_exceed(ktau, X, ident) == 3)
    assert full.shape == (P,)


def test_pvalues_and_errors(ktau):
    X = uniform_ties(30, 40, seed=23)
    perms = permutations(9, 40, seed=24)
    res = ktau.permutation_pvalues(torch.from_numpy(X).cuda(), torch.from_numpy(perms))
    ref = oracle.permutation_exceed(X, perms)
    assert np.array_equal(res["exceed"].cpu().numpy().astype(np.int64), ref)
    # (exceed + 1) / (B + 1): the IEEE FP64 quotient, computed by the library
    assert np.array_equal(res["pvalue"].cpu().numpy(), (ref + 1) / 10.0)
    res["ranked"].free()
    Xl = torch.from_numpy(uniform_ties(10, 5793, seed=25)).cuda()  # beyond the contraction
    R = ktau.ktau_rank_prepare(Xl)
    S = torch.zeros(45, dtype=torch.int32, device="cuda")
    exc = torch.zeros(45, dtype=torch.uint32, device="cuda")
    with pytest.raises(ktau.KtauError):
        ktau.ktau_permutation_exceed(R, torch.from_numpy(permutations(2, 5793)).cuda(), S, exc)
    with pytest.raises(ValueError):
        ktau.ktau_permutation_exceed(R, torch.zeros((2, 5), dtype=torch.int32, device="cuda"),
                                     S, exc)
    R.free()
