"""Parity of the Knight merge path (K-a rank kernel + K-b count kernel) with the CPU oracle:
exact integer counts (S = n_c - n_d, n_3), tau-b within 1e-12 relative, FP32 = RN(FP64)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import assert_tau32, assert_tau64, oracle_full, oracle_sampled
from synthetic import gene_expression, heavy_ties_ordinal, uniform_ties

pytestmark = pytest.mark.gpu

MERGE = {"path": 1}


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _run(ktau, X, count_bits=32, options=MERGE, p_begin=0, p_end=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    res = ktau.allpairs(Xd, p_begin=p_begin, p_end=p_end, count_bits=count_bits,
                        options=options)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    return out


def _check(got, ref):
    assert np.array_equal(got["S"].astype(np.int64), ref["S"])
    assert np.array_equal(got["n3"].astype(np.int64), ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


@pytest.mark.parametrize("count_bits", [32, 64])
def test_uniform_ties_64x200_all_pairs(ktau, count_bits):
    X = uniform_ties(64, 200, seed=0)
    got = _run(ktau, X, count_bits)
    ref = oracle_full(X)
    _check(got, ref)
    assert got["S"].size == 2016
    assert got["T"].shape == (64,)


@pytest.mark.parametrize("n", [2, 5, 31, 32, 33, 64, 97, 128, 200, 255, 256, 257, 1000])
@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_tie_counts_and_ranks(ktau, n, dtype):
    m = 45 if n <= 256 else 12  # ragged against the eight variables of a rank CTA
    X = uniform_ties(m, n, tie_frac=0.3, seed=4 + n)
    if dtype == "i32":
        X = np.floor(X * 7).astype(np.int32) - 3
    else:
        X[0, 0], X[0, -1] = -0.0, 0.0  # equal values
        X[1, 0], X[1, -1] = np.inf, -np.inf
        X[2, :] = 1.5  # one tie group
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    T = ktau.ktau_tie_counts(R).cpu().numpy()
    perm, rank = ktau.ktau_ranked_export(R)
    perm = perm.cpu().numpy().astype(np.int64)
    rank = rank.cpu().numpy().astype(np.int64)
    R.free()
    for i in range(X.shape[0]):
        p, r, t = oracle.rank(X[i])
        assert np.array_equal(perm[i], p)
        assert np.array_equal(rank[i], r)
        assert T[i] == t


@pytest.mark.parametrize("n", [2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 255, 256,
                               257, 300, 1000, 2049])
@pytest.mark.parametrize("mapping", [1, 2])
def test_ragged_n(ktau, n, mapping):
    m = 70 if n <= 300 else 20
    X = uniform_ties(m, n, tie_frac=0.3, seed=n)
    X[3] = X[5]  # duplicated row
    if n > 4:
        X[7, : n // 2] = 0.5  # a heavy tie group
    got = _run(ktau, X, 64, options={"path": 1, "mapping": mapping, "tile_q": 16 if n < 100 else 0})
    _check(got, oracle_full(X))


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("tile_q", [1, 5, 32, 64])
def test_tiles_and_schedules(ktau, schedule, tile_q):
    X = uniform_ties(75, 48, seed=tile_q)
    got = _run(ktau, X, 32, options={"path": 1, "tile_q": tile_q, "schedule": schedule})
    _check(got, oracle_full(X))


def test_ranges_concatenate(ktau):
    """Multi-pass sub-ranges (Sec. 4.3.1) give exactly the slices of one full launch."""
    X = uniform_ties(53, 77, seed=3)
    P = 53 * 52 // 2
    full = _run(ktau, X, 64)
    cuts = [0, 1, 2, 51, 52, 300, 999, P - 1, P]
    for a, b in zip(cuts, cuts[1:]):
        part = _run(ktau, X, 64, p_begin=a, p_end=b)
        assert np.array_equal(part["S"], full["S"][a:b])
        assert np.array_equal(part["n3"], full["n3"][a:b])
        assert np.array_equal(part["tau64"].view(np.int64), full["tau64"][a:b].view(np.int64))


def test_edge_values(ktau):
    n = 40
    X = np.random.default_rng(0).random((6, n)).astype(np.float32)
    X[0] = 1.0  # constant row -> NaN tau for every pair that contains it
    X[1, :3] = [np.inf, -np.inf, np.inf]
    X[2, :4] = [-0.0, 0.0, -0.0, 0.0]
    X[3] = -X[2]
    X[4] = X[1][::-1]
    got = _run(ktau, X, 64)
    ref = oracle_full(X)
    _check(got, ref)
    assert np.isnan(got["tau64"][:5]).all()


def test_two_rows_and_int32(ktau):
    X = np.array([[3, 1, 4, 1, 5], [9, 2, 6, 5, 3]], np.int32)
    got = _run(ktau, X, 32)
    assert got["S"].tolist() == [1] and got["n3"].tolist() == [0]
    assert got["tau64"][0] == 1 / np.sqrt(90.0)
    Xi = heavy_ties_ordinal(m=30, n=301, seed=2)
    _check(_run(ktau, Xi, 64), oracle_full(Xi))


def test_all_rows_constant(ktau):
    X = np.full((5, 17), 2.0, np.float32)
    got = _run(ktau, X, 32)
    assert (got["S"] == 0).all() and np.isnan(got["tau64"]).all()
    assert (got["n3"] == 17 * 16 // 2).all()


def test_nan_rejected(ktau):
    X = np.random.default_rng(1).random((4, 10)).astype(np.float32)
    X[2, 7] = np.nan
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_rank_prepare(torch.from_numpy(X).cuda())
    assert ei.value.status == 2


def test_max_n(ktau):
    n = ktau.KTAU_NARROW_MAX_N  # the longest rows kept with 16-bit ranks
    X = heavy_ties_ordinal(m=3, n=n, levels=5000, seed=1)
    got = _run(ktau, X, 64, options={"path": 1, "mapping": 2})
    _check(got, oracle_full(X))


def test_gene_expression_full_size_sampled(ktau):
    """The benchmark workload: m=16384 x n=128, packed FP32 tau + int32 counts, merge path."""
    X = gene_expression(16384, 128, seed=0)
    m = X.shape[0]
    P = m * (m - 1) // 2
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    tau32 = torch.empty(P, dtype=torch.float32, device="cuda")
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    n3 = torch.empty(P, dtype=torch.int32, device="cuda")
    ktau.ktau_allpairs(R, 0, P, None, tau32, S, n3, 32, MERGE)
    torch.cuda.synchronize()
    g = np.random.default_rng(0)
    ps = np.unique(np.concatenate([g.integers(0, P, 3000), [0, 1, P - 2, P - 1],
                                   np.arange(16383, 16383 + 64)]))
    idx = torch.from_numpy(ps).cuda()
    rS, rn3, rtau = oracle_sampled(X, ps)
    assert np.array_equal(S[idx].cpu().numpy().astype(np.int64), rS)
    assert np.array_equal(n3[idx].cpu().numpy().astype(np.int64), rn3)
    assert_tau32(tau32[idx].cpu().numpy(), rtau)
    # every pair was written: tau in [-1, 1], S within +-n_0
    t = tau32.cpu().numpy()
    assert np.isfinite(t).all() and np.abs(t).max() <= 1.0
    R.free()


def test_heavy_ties_full_size_sampled(ktau):
    """Long heavy-tie profiles: m=2048 x n=4096 int32 in 0..63, int64 counts, FP64 tau."""
    X = heavy_ties_ordinal(2048, 4096, seed=0)
    m = X.shape[0]
    P = m * (m - 1) // 2
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    tau = torch.empty(P, dtype=torch.float64, device="cuda")
    S = torch.empty(P, dtype=torch.int64, device="cuda")
    n3 = torch.empty(P, dtype=torch.int64, device="cuda")
    ktau.ktau_allpairs(R, 0, P, tau, None, S, n3, 64, MERGE)
    torch.cuda.synchronize()
    g = np.random.default_rng(1)
    ps = np.unique(np.concatenate([g.integers(0, P, 600), [0, P - 1]]))
    idx = torch.from_numpy(ps).cuda()
    rS, rn3, rtau = oracle_sampled(X, ps)
    assert np.array_equal(S[idx].cpu().numpy(), rS)
    assert np.array_equal(n3[idx].cpu().numpy(), rn3)
    assert_tau64(tau[idx].cpu().numpy(), rtau)
    R.free()
