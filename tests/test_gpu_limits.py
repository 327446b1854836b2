"""Edge cases at the limits of the ABI: the longest vectors on the merge path (rows beyond
16384 samples are ranked in chunks merged in global scratch and counted with global merge
buffers; n = 65535 is the longest kept with 16-bit ranks, longer rows keep 32-bit ranks and
64-bit merge keys), a large matrix (300,000 variables) with a pair range at the end of the
triangle on both paths (64-bit pair indices, tile walks far from the origin), and inputs just
beyond the limits."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_tau32, assert_tau64, oracle_full, oracle_sampled
from synthetic import heavy_ties_ordinal, uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


@pytest.mark.parametrize("n", [16384, 16385, 40000, 65535])
def test_longest_vectors_merge_path(ktau, n):
    X = uniform_ties(5, n, tie_frac=0.3, seed=31)
    X[1] = X[0]
    X[2] = -X[0]
    Xd = torch.from_numpy(X).cuda()
    res = ktau.allpairs(Xd, count_bits=64, options={"path": 1})
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    got = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    ref = oracle_full(X)
    assert np.array_equal(got["S"], ref["S"])
    assert np.array_equal(got["n3"], ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


@pytest.mark.parametrize("path", [1, 2])
def test_large_matrix_tail_range(ktau, path):
    m, n = 300_000, 32
    X = uniform_ties(m, n, tie_frac=0.3, seed=32)
    X[m - 1] = X[m - 2]
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    P = m * (m - 1) // 2
    lo, hi = P - 70_000, P
    tau64 = torch.empty(hi - lo, dtype=torch.float64, device="cuda")
    tau32 = torch.empty(hi - lo, dtype=torch.float32, device="cuda")
    S = torch.empty(hi - lo, dtype=torch.int64, device="cuda")
    n3 = torch.empty(hi - lo, dtype=torch.int64, device="cuda")
    ktau.ktau_allpairs(R, lo, hi, tau64, tau32, S, n3, 64, {"path": path})
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    R.free()
    g = np.random.default_rng(33)
    ps = np.unique(np.concatenate([g.integers(lo, hi, 400), [lo, hi - 1]]))
    rS, rn3, rtau = oracle_sampled(X, ps)
    idx = ps - lo
    assert np.array_equal(S.cpu().numpy()[idx], rS)
    assert np.array_equal(n3.cpu().numpy()[idx], rn3)
    assert_tau64(tau64.cpu().numpy()[idx], rtau)
    assert_tau32(tau32.cpu().numpy()[idx], rtau)


@pytest.mark.parametrize("n", [20000, 65535])
def test_long_rows_ranks_and_async(ktau, n):
    """Long-row rank transform (chunks merged in global scratch) against the oracle's ranks, through
    the synchronous and the asynchronous prepare, integer values with heavy ties."""
    import oracle

    g = np.random.default_rng(n)
    X = g.integers(-50, 50, (3, n)).astype(np.int32)
    X[1] = np.arange(n)[::-1]  # no ties, reversed
    Xd = torch.from_numpy(X).cuda()
    for fn in (ktau.ktau_rank_prepare, ktau.ktau_rank_prepare_async):
        R = fn(Xd)
        perm, rank = ktau.ktau_ranked_export(R)
        T = ktau.ktau_tie_counts(R).cpu().numpy()
        torch.cuda.synchronize()
        for i in range(3):
            p, r, t = oracle.rank(X[i].astype(np.float64))
            assert np.array_equal(perm[i].cpu().numpy().astype(np.int64), p)
            assert np.array_equal(rank[i].cpu().numpy().astype(np.int64), r)
            assert T[i] == t
        R.free()


def test_long_rows_query(ktau):
    """Query search with long profiles (n > 16384): merge path with global merge buffers."""
    import oracle

    n = 20000
    D = uniform_ties(7, n, tie_frac=0.2, seed=41)
    Q = uniform_ties(2, n, tie_frac=0.2, seed=42)
    Q[1] = D[3]
    db = ktau.ktau_rank_prepare(torch.from_numpy(D).cuda())
    q = ktau.ktau_rank_prepare(torch.from_numpy(Q).cuda())
    S = torch.empty((2, 7), dtype=torch.int64, device="cuda")
    n3 = torch.empty((2, 7), dtype=torch.int64, device="cuda")
    tau = torch.empty((2, 7), dtype=torch.float64, device="cuda")
    idx = torch.empty((2, 3), dtype=torch.int32, device="cuda")
    tk = torch.empty((2, 3), dtype=torch.float64, device="cuda")
    ktau.ktau_query(db, q, tau, S, n3, 64, 3, idx, tk)
    torch.cuda.synchronize()
    ref = oracle.query_topk(Q, D, 3)
    assert np.array_equal(S.cpu().numpy(), ref["S"])
    assert np.array_equal(n3.cpu().numpy(), ref["n3"])
    assert_tau64(tau.cpu().numpy().ravel(), ref["tau"].ravel())
    assert np.array_equal(idx.cpu().numpy(), ref["topk_idx"])
    db.free()
    q.free()


@pytest.mark.parametrize("n,dtype", [(65536, "f32"), (70001, "i32"), (100003, "f32"),
                                     ((1 << 20) + 3, "i32")])
def test_wide_rows_merge_path(ktau, n, dtype):
    """Rows longer than 65535 samples: 32-bit ranks, Step 1 keys (group << 32 | w) in 64 bits,
    counts with 64-bit accumulators. Float rows with 30% ties and exact copies / negations;
    integer rows with about 5000 tie groups (Step 1 stops early and fixes up)."""
    if dtype == "f32":
        X = uniform_ties(4, n, tie_frac=0.3, seed=n)
    else:
        X = heavy_ties_ordinal(m=4, n=n, levels=5000, seed=n)
    X[1] = X[0]
    X[2] = -X[0]
    Xd = torch.from_numpy(X).cuda()
    res = ktau.allpairs(Xd, count_bits=64, options={"path": 1})
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    got = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    ref = oracle_full(X)
    assert np.array_equal(got["S"], ref["S"])
    assert np.array_equal(got["n3"], ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


def test_wide_rows_ranks_and_range(ktau):
    """32-bit ranks against the oracle's (both prepare forms), a sub-range of the triangle, and
    every form that keeps 16-bit ranks refusing the handle."""
    import oracle

    n = 70000
    g = np.random.default_rng(5)
    X = g.integers(-3000, 3000, (5, n)).astype(np.int32)
    X[3] = np.arange(n)[::-1]
    Xd = torch.from_numpy(X).cuda()
    for fn in (ktau.ktau_rank_prepare, ktau.ktau_rank_prepare_async):
        R = fn(Xd)
        perm, rank = ktau.ktau_ranked_export32(R)
        T = ktau.ktau_tie_counts(R).cpu().numpy()
        torch.cuda.synchronize()
        for i in range(5):
            p, r, t = oracle.rank(X[i].astype(np.float64))
            assert np.array_equal(perm[i].cpu().numpy().astype(np.int64), p)
            assert np.array_equal(rank[i].cpu().numpy().astype(np.int64), r)
            assert T[i] == t
        R.free()
    R = ktau.ktau_rank_prepare(Xd)
    lo, hi = 3, 9
    S = torch.empty(hi - lo, dtype=torch.int64, device="cuda")
    n3 = torch.empty(hi - lo, dtype=torch.int64, device="cuda")
    ktau.ktau_allpairs(R, lo, hi, None, None, S, n3, 64, None)
    torch.cuda.synchronize()
    ref = oracle_full(X)
    assert np.array_equal(S.cpu().numpy(), ref["S"][lo:hi])
    assert np.array_equal(n3.cpu().numpy(), ref["n3"][lo:hi])
    S32 = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:  # n_0 >= 2^31: 64-bit counts only
        ktau.ktau_allpairs(R, lo, hi, None, None, S32, None, 32, None)
    assert ei.value.status == 3
    for opts in ({"path": 2}, {"path": 3}, {"path": 1, "mapping": 1}):
        with pytest.raises(ktau.KtauError) as ei:
            ktau.ktau_allpairs(R, lo, hi, None, None, S, None, 64, opts)
        assert ei.value.status == 1
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_ranked_export(R)
    assert ei.value.status == 1
    Sq = torch.empty((5, 5), dtype=torch.int64, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_query(R, R, None, Sq, None, 64)
    assert ei.value.status == 3
    R.free()


def test_longest_rows(ktau):
    """n = KTAU_MAX_N (4,194,304 samples): ranks through six global merge levels, 64-bit keys,
    S up to n_0 ~ 8.8e12 (tau32 from the FP64 formula above 2^31)."""
    n = ktau.KTAU_MAX_N
    g = np.random.default_rng(9)
    X = g.standard_normal((3, n)).astype(np.float32)
    X[1] = X[0]
    X[2] = np.round(X[0] * 4) / 4  # heavy ties, monotone in row 0
    Xd = torch.from_numpy(X).cuda()
    res = ktau.allpairs(Xd, count_bits=64, options={"path": 1})
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    got = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    del Xd
    torch.cuda.empty_cache()
    ref = oracle_full(X)
    assert np.array_equal(got["S"], ref["S"])
    assert np.array_equal(got["n3"], ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


def test_export32_of_short_rows(ktau):
    """ktau_ranked_export32 on a 16-bit handle widens its rows."""
    X = uniform_ties(3, 300, tie_frac=0.3, seed=7)
    R = ktau.ktau_rank_prepare(torch.from_numpy(X).cuda())
    p16, r16 = ktau.ktau_ranked_export(R)
    p32, r32 = ktau.ktau_ranked_export32(R)
    torch.cuda.synchronize()
    assert np.array_equal(p16.cpu().numpy().astype(np.int64), p32.cpu().numpy())
    assert np.array_equal(r16.cpu().numpy().astype(np.int64), r32.cpu().numpy())
    R.free()


def test_beyond_limits_rejected(ktau):
    X = torch.zeros((2, ktau.KTAU_MAX_N + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_rank_prepare(X)
    assert ei.value.status == 3
    # the batched and allocation-free forms stop at n = 16384
    Xb = torch.zeros((2, 16385), dtype=torch.float32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.Batch([ktau.batch_desc(Xb)])
    assert ei.value.status == 3
    Sb = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_allpairs_noalloc(Xb, 0, 1, None, None, Sb, None, 32)
    assert ei.value.status == 3
    X = torch.zeros((3, 1), dtype=torch.float32, device="cuda")  # n < 2
    with pytest.raises(ktau.KtauError):
        ktau.ktau_rank_prepare(X)
    Xd = torch.from_numpy(uniform_ties(10, 5793, seed=34)).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    out = torch.empty(45, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError):  # sign contraction: n <= 5792 (n_0 < 2^24)
        ktau.ktau_allpairs(R, 0, 45, None, None, out, None, 32, {"path": 2})
    R.free()
    Xd = torch.from_numpy(uniform_ties(10, 3001, seed=35)).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    n3 = torch.empty(45, dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError) as ei:  # n_3 beyond 3000 samples: FP4 operands only
        ktau.ktau_allpairs(R, 0, 45, None, None, out, n3, 32, {"path": 2, "operand_bits": 8})
    assert ei.value.status == 1
    R.free()
