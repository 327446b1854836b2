"""Query form: exact tau-b of every query profile against every database variable, plus the
exact top-k by |tau| (ties -> smaller row index, NaN last), against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import assert_tau64
from synthetic import gene_expression, uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _query(ktau, Q, D, k, path=0, count_bits=32, bits=0):
    Rq = ktau.ktau_rank_prepare(torch.from_numpy(np.ascontiguousarray(Q)).cuda())
    Rd = ktau.ktau_rank_prepare(torch.from_numpy(np.ascontiguousarray(D)).cuda())
    b, m = Q.shape[0], D.shape[0]
    cdt = torch.int32 if count_bits == 32 else torch.int64
    tau = torch.empty((b, m), dtype=torch.float64, device="cuda")
    S = torch.empty((b, m), dtype=cdt, device="cuda")
    n3 = torch.empty((b, m), dtype=cdt, device="cuda")
    idx = torch.empty((b, max(k, 1)), dtype=torch.int32, device="cuda")
    tk = torch.empty((b, max(k, 1)), dtype=torch.float64, device="cuda")
    ktau.ktau_query(Rd, Rq, tau, S, n3, count_bits, k, idx, tk,
                    {"path": path, "operand_bits": bits})
    ktau.ktau_device_status()
    out = {"tau": tau.cpu().numpy(), "S": S.cpu().numpy().astype(np.int64),
           "n3": n3.cpu().numpy().astype(np.int64), "idx": idx.cpu().numpy()[:, :k],
           "tk": tk.cpu().numpy()[:, :k]}
    Rq.free()
    Rd.free()
    return out


def _check(got, Q, D, k):
    ref = oracle.query_topk(Q, D, k)
    assert np.array_equal(got["S"], ref["S"])
    assert np.array_equal(got["n3"], ref["n3"])
    assert_tau64(got["tau"].ravel(), ref["tau"].ravel())
    assert np.array_equal(got["idx"], ref["topk_idx"])
    assert_tau64(got["tk"].ravel(), ref["topk_tau"].ravel())


@pytest.mark.parametrize("n,path,bits", [(100, 0, 0), (200, 0, 0), (100, 1, 0), (1100, 0, 0),
                                         (60, 2, 0), (200, 2, 4), (1100, 2, 4)])
def test_query_matches_oracle(ktau, n, path, bits):
    D = uniform_ties(300 if n < 1000 else 120, n, tie_frac=0.3, seed=n)
    D[10] = D[11]          # exact |tau| ties -> index order
    D[12] = -D[11]
    D[20] = 0.5            # constant database row -> NaN, ranked last
    Q = uniform_ties(7, n, tie_frac=0.3, seed=n + 1)
    Q[2] = D[11]
    k = 50
    _check(_query(ktau, Q, D, k, path, bits=bits), Q, D, k)


def test_full_sort_and_constant_query(ktau):
    D = uniform_ties(130, 40, tie_frac=0.5, seed=3)
    D[5] = 1.0
    Q = uniform_ties(4, 40, tie_frac=0.5, seed=4)
    Q[1] = 2.0  # constant query: every tau NaN, order = row index
    for k in (1, 7, 130):
        got = _query(ktau, Q, D, k)
        _check(got, Q, D, k)
    assert list(got["idx"][1]) == list(range(130))


def test_count_bits_64_and_no_outputs(ktau):
    D = uniform_ties(200, 90, seed=8)
    Q = uniform_ties(5, 90, seed=9)
    _check(_query(ktau, Q, D, 20, count_bits=64), Q, D, 20)
    # top-k only (the library uses its own scratch for S)
    Rq = ktau.ktau_rank_prepare(torch.from_numpy(Q).cuda())
    Rd = ktau.ktau_rank_prepare(torch.from_numpy(D).cuda())
    idx = torch.empty((5, 20), dtype=torch.int32, device="cuda")
    tk = torch.empty((5, 20), dtype=torch.float64, device="cuda")
    ktau.ktau_query(Rd, Rq, None, None, None, 32, 20, idx, tk)
    ref = oracle.query_topk(Q, D, 20)
    assert np.array_equal(idx.cpu().numpy(), ref["topk_idx"])


def test_sample_count_mismatch(ktau):
    Rq = ktau.ktau_rank_prepare(torch.rand((3, 50), device="cuda"))
    Rd = ktau.ktau_rank_prepare(torch.rand((30, 51), device="cuda"))
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_query(Rd, Rq, None, None, None, 32, 0, None, None)
    assert ei.value.status == 1


def test_resident_database_full_size(ktau):
    """Serving-sized database: 65536 x 256 gene-expression profiles, 48 queries, top-100."""
    D = gene_expression(65536, 256, seed=0)
    Q = gene_expression(48, 256, seed=1)
    Rd = ktau.ktau_rank_prepare(torch.from_numpy(D).cuda())
    Rq = ktau.ktau_rank_prepare(torch.from_numpy(Q).cuda())
    b, m, k = 48, 65536, 100
    S = torch.empty((b, m), dtype=torch.int32, device="cuda")
    tau = torch.empty((b, m), dtype=torch.float64, device="cuda")
    idx = torch.empty((b, k), dtype=torch.int32, device="cuda")
    tk = torch.empty((b, k), dtype=torch.float64, device="cuda")
    ktau.ktau_query(Rd, Rq, tau, S, None, 32, k, idx, tk)
    ktau.ktau_device_status()
    g = np.random.default_rng(0)
    Sh = S.cpu().numpy()
    taus = tau.cpu().numpy()
    for q in g.choice(b, 6, replace=False):
        js = g.choice(m, 300, replace=False)
        for j in js[:60]:
            c = oracle.pair_counts(Q[q].astype(np.float64), D[j].astype(np.float64), "knight")
            assert Sh[q, j] == c["S"]
    # exact top-k of two queries against the oracle's full row
    for q in (0, 17):
        ref = oracle.query_topk(Q[q:q + 1], D, k)
        assert np.array_equal(idx[q].cpu().numpy(), ref["topk_idx"][0])
        assert_tau64(tk[q].cpu().numpy(), ref["topk_tau"][0])
        assert_tau64(taus[q], ref["tau"][0])
    Rq.free()
    Rd.free()


@pytest.mark.parametrize("k", [1, 100, 1024])
def test_topk_across_chunks_with_duplicate_rows(ktau, k):
    """Top-k over a database of 20000 rows in several chunks of 4096: rows repeated every 4096
    (exactly equal |tau| in different chunks, broken by the smaller row index), a row negated,
    k = 1024 takes two candidate passes before the final one."""
    D = gene_expression(20000, 64, seed=3)
    for c in range(1, 5):
        hi = min(20000, 4096 * (c + 1))
        D[4096 * c:hi] = D[:hi - 4096 * c]
    D[19999] = -D[5]
    Q = gene_expression(3, 64, seed=4)
    Q[2] = D[5]
    Rd = ktau.ktau_rank_prepare(torch.from_numpy(D).cuda())
    Rq = ktau.ktau_rank_prepare(torch.from_numpy(Q).cuda())
    b, m = 3, 20000
    S = torch.empty((b, m), dtype=torch.int32, device="cuda")
    idx = torch.empty((b, k), dtype=torch.int32, device="cuda")
    tk = torch.empty((b, k), dtype=torch.float64, device="cuda")
    ktau.ktau_query(Rd, Rq, None, S, None, 32, k, idx, tk)
    ktau.ktau_device_status()
    ref = oracle.query_topk(Q, D, k)
    assert np.array_equal(idx.cpu().numpy(), ref["topk_idx"])
    assert_tau64(tk.cpu().numpy().ravel(), ref["topk_tau"].ravel())
    Rq.free()
    Rd.free()
