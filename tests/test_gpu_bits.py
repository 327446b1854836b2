"""Bit-parallel dominance count (KTAU_PATH_BITS): the sign form of Algorithm 1 over per-sample
masks of larger / smaller ranks. Exact counts against the oracle for every short n (one and
several mask words, ragged tails), constant / duplicated / reversed rows and heavy ties;
bit-identical to the merge path on the full 16384 x 128 workload; sub-ranges, tau-a, limits."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_tau32, assert_tau64, oracle_full
from synthetic import gene_expression, heavy_ties_ordinal, uniform_ties

pytestmark = pytest.mark.gpu

BITS = {"path": 3}


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _run(ktau, X, count_bits=64, options=BITS, p_begin=0, p_end=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    res = ktau.allpairs(Xd, p_begin=p_begin, p_end=p_end, count_bits=count_bits, options=options)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    return out


@pytest.mark.parametrize("n", [2, 3, 5, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200,
                               255, 256])
def test_matches_oracle(ktau, n):
    m = 70 if n > 100 else 90  # several 16-variable tiles, ragged
    X = uniform_ties(m, n, tie_frac=0.3, seed=n)
    X[3] = X[4]          # duplicated variable: S = n_0 - T
    X[5] = -X[4]         # reversed
    X[6] = 0.5           # constant variable: tau NaN
    X[7, : n // 2] = 2.0
    got = _run(ktau, X)
    ref = oracle_full(X)
    assert np.array_equal(got["S"], ref["S"])
    assert np.array_equal(got["n3"], ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


def test_heavy_ties_and_ranges(ktau):
    X = heavy_ties_ordinal(m=120, n=150, levels=6, seed=3)
    P = 120 * 119 // 2
    full = _run(ktau, X, 32)
    ref = oracle_full(X)
    assert np.array_equal(full["S"].astype(np.int64), ref["S"])
    assert np.array_equal(full["n3"].astype(np.int64), ref["n3"])
    for lo, hi in ((0, 1), (17, 4000), (P - 300, P)):
        part = _run(ktau, X, 32, p_begin=lo, p_end=hi)
        for k in ("S", "n3", "tau64", "tau32"):
            a, b = part[k], full[k][lo:hi]
            assert np.array_equal(a.view(np.int64 if a.itemsize == 8 else np.int32),
                                  b.view(np.int64 if b.itemsize == 8 else np.int32)), k


def test_full_size_identical_to_merge_path(ktau):
    """The 16384 x 128 workload: every output bit-identical to the merge path's."""
    X = gene_expression(16384, 128, seed=0)
    a = _run(ktau, X, 32, options=BITS)
    b = _run(ktau, X, 32, options={"path": 1})
    for k in ("S", "n3", "tau32"):
        assert np.array_equal(a[k].view(np.int32), b[k].view(np.int32)), k


def test_tau_a_and_limits(ktau):
    X = uniform_ties(40, 90, tie_frac=0.2, seed=9)
    got = _run(ktau, X, 32, options={"path": 3, "statistic": 1})
    ref = _run(ktau, X, 32, options={"path": 1, "statistic": 1})
    assert np.array_equal(got["tau32"].view(np.int32), ref["tau32"].view(np.int32))
    assert np.array_equal(got["tau64"].view(np.int64), ref["tau64"].view(np.int64))
    with pytest.raises(ktau.KtauError):  # n > KTAU_BITS_MAX_N
        _run(ktau, uniform_ties(5, 257, seed=1), 32)
    Xd = torch.from_numpy(uniform_ties(6, 40, seed=2)).cuda()
    db = ktau.ktau_rank_prepare(Xd)
    S = torch.empty((6, 6), dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError):  # triangle of one matrix only
        ktau.ktau_query(db, db, None, S, None, 32, 0, None, None, BITS)
    db.free()
