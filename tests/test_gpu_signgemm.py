"""Parity of the tensor-core sign contraction (K-c) with the CPU oracle, and bit-identity with
the merge path (K-b): both form tau-b through the same epilogue from exact integer counts."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_tau32, assert_tau64, oracle_full, oracle_sampled
from synthetic import gene_expression, heavy_ties_ordinal, uniform_ties

pytestmark = pytest.mark.gpu

SG = {"path": 2}
MERGE = {"path": 1}


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _run(ktau, X, count_bits=32, options=SG, p_begin=0, p_end=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    res = ktau.allpairs(Xd, p_begin=p_begin, p_end=p_end, count_bits=count_bits, options=options)
    torch.cuda.synchronize()
    ktau.ktau_device_status()  # a bounded wait that gave up raises here
    out = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    return out


def _check(got, ref):
    assert np.array_equal(got["S"].astype(np.int64), ref["S"])
    assert np.array_equal(got["n3"].astype(np.int64), ref["n3"])
    assert_tau64(got["tau64"], ref["tau"])
    assert_tau32(got["tau32"], ref["tau"])


@pytest.mark.parametrize("bits", [4, 8, 16])
def test_uniform_ties_64x200(ktau, bits):
    X = uniform_ties(64, 200, seed=0)
    _check(_run(ktau, X, 64, options={"path": 2, "operand_bits": bits}), oracle_full(X))


@pytest.mark.parametrize("bits", [0, 4])
@pytest.mark.parametrize("n", [2, 3, 5, 8, 9, 15, 16, 17, 64, 100, 127, 128, 129, 200, 256, 300,
                               1100])
def test_ragged(ktau, n, bits):
    m = 300 if n < 1000 else 90  # two 256-row super-tiles, ragged
    X = uniform_ties(m, n, tie_frac=0.2, seed=n)
    X[10] = X[11]
    X[12] = -X[13]
    X[20, : n // 2] = 0.25
    _check(_run(ktau, X, 32, options={"path": 2, "operand_bits": bits}), oracle_full(X))


@pytest.mark.parametrize("n,bits", [(128, 8), (256, 8), (512, 8), (1024, 8), (2048, 8),
                                    (2900, 8), (256, 16), (128, 4), (300, 4), (1024, 4),
                                    (2048, 4), (4096, 4), (5792, 4)])
def test_extreme_counts(ktau, n, bits):
    """Exactness of the tensor-core sums: |S| = n_0 (identical and reversed rows, the largest
    partial sums), and strongly correlated rows, whose partial sums grow large while each MMA adds
    a small, irregular increment (any truncation of the FP32 accumulator would show here)."""
    g = np.random.default_rng(n)
    base = g.random(n).astype(np.float32)
    rows = [base, base, -base, base * 2 + 1, g.random(n).astype(np.float32)]
    rows += [(base + 0.05 * g.random(n)).astype(np.float32) for _ in range(12)]
    X = np.stack(rows * (2 if n >= 1024 else (3 if n >= 512 else 8)))
    got = _run(ktau, X, 64, options={"path": 2, "operand_bits": bits})
    ref = oracle_full(X)
    _check(got, ref)
    n0 = n * (n - 1) // 2
    assert got["S"].max() == n0 and got["S"].min() == -n0


def test_ranges_and_large_m(ktau):
    X = uniform_ties(1000, 60, seed=5)
    P = 1000 * 999 // 2
    full = _run(ktau, X, 32)
    g = np.random.default_rng(2)
    ps = np.unique(np.concatenate([g.integers(0, P, 500), [0, P - 1]]))
    rS, rn3, rtau = oracle_sampled(X, ps)
    assert np.array_equal(full["S"][ps].astype(np.int64), rS)
    assert np.array_equal(full["n3"][ps].astype(np.int64), rn3)
    for a, b in [(0, 1), (5, 70000), (123456, 123457), (P - 1000, P)]:
        part = _run(ktau, X, 32, p_begin=a, p_end=b)
        assert np.array_equal(part["S"], full["S"][a:b])
        assert np.array_equal(part["tau32"].view(np.int32), full["tau32"][a:b].view(np.int32))


def test_constant_and_tied_rows(ktau):
    X = uniform_ties(40, 90, tie_frac=0.5, seed=9)
    X[0] = 3.0
    X[1, :45] = 1.0
    X[2] = np.round(X[2] * 3)
    _check(_run(ktau, X, 32), oracle_full(X))


def test_gene_expression_matches_merge_bitwise(ktau):
    """Benchmark workload: the whole packed triangle of both paths is bit-identical, and
    sampled pairs match the oracle."""
    X = gene_expression(16384, 128, seed=0)
    m = X.shape[0]
    P = m * (m - 1) // 2
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    outs = {}
    for name, opt in (("sg", SG), ("sg4", {"path": 2, "operand_bits": 4}), ("merge", MERGE)):
        tau32 = torch.empty(P, dtype=torch.float32, device="cuda")
        S = torch.empty(P, dtype=torch.int32, device="cuda")
        n3 = torch.empty(P, dtype=torch.int32, device="cuda")
        ktau.ktau_allpairs(R, 0, P, None, tau32, S, n3, 32, opt)
        outs[name] = (tau32, S, n3)
    torch.cuda.synchronize()
    for a, b, c in zip(outs["sg"], outs["sg4"], outs["merge"]):
        assert torch.equal(a.view(torch.int32), c.view(torch.int32))
        assert torch.equal(b.view(torch.int32), c.view(torch.int32))
    g = np.random.default_rng(0)
    ps = np.unique(np.concatenate([g.integers(0, P, 2000), [0, P - 1]]))
    idx = torch.from_numpy(ps).cuda()
    rS, rn3, rtau = oracle_sampled(X, ps)
    tau32, S, n3 = outs["sg"]
    assert np.array_equal(S[idx].cpu().numpy().astype(np.int64), rS)
    assert np.array_equal(n3[idx].cpu().numpy().astype(np.int64), rn3)
    assert_tau32(tau32[idx].cpu().numpy(), rtau)
    R.free()


@pytest.mark.parametrize("dups", [0, 1, 3])
def test_joint_ties_bucket_and_tile_forms(ktau, dups):
    """n_3 on the triangle: with few shared ties the inverted-index (bucket) form counts it; when
    `dups` sample columns repeat another column in every variable, a tied sample pair is shared
    by all 760 variables (one bucket of 288,420 pairs), so the tile form counts it instead. Both
    must agree with the oracle exactly, also on sub-ranges."""
    m, n = 760, 96
    X = uniform_ties(m, n, tie_frac=0.1, seed=40 + dups)
    for d in range(dups):
        X[:, 2 * d + 1] = X[:, 2 * d]
    ref = oracle_full(X)
    _check(_run(ktau, X, 32), ref)
    P = m * (m - 1) // 2
    lo, hi = P // 3 + 5, P // 3 + 20000
    got = _run(ktau, X, 64, p_begin=lo, p_end=hi)
    assert np.array_equal(got["n3"].astype(np.int64), ref["n3"][lo:hi])
    assert np.array_equal(got["S"].astype(np.int64), ref["S"][lo:hi])


@pytest.mark.parametrize("n,m", [(300, 60), (3000, 24), (5792, 8)])
def test_heavy_ties_magnitude_contraction(ktau, n, m):
    """Tie-heavy long profiles (64 values per variable, about n^2/128 tied sample pairs each) on
    the default path: S from the sign contraction, n_3 from the contraction of the magnitudes
    (|A_u| . |A_v| = n_0 - T_u - T_v + n_3), checked against the oracle element by element."""
    X = heavy_ties_ordinal(m=m, n=n, levels=64, seed=n)
    X[1] = X[0]
    X[2] = 63 - X[0]
    got = _run(ktau, X, 64, options=None)
    _check(got, oracle_full(X))
    R = ktau.ktau_rank_prepare(torch.from_numpy(X).cuda())
    assert ktau.ktau_allpairs_path(R) == 2  # the contraction is the default for these rows
    R.free()
