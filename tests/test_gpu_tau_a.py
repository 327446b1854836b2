"""tau-a (Sec. 2: (n_c - n_d) / n_0, no tie correction) on both pair paths: FP64 output equal to
the IEEE quotient S / n_0, FP32 output equal to S / n_0 correctly rounded, bit for bit, against
the oracle; forms that compute tau-b only reject the option."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import oracle_full
from synthetic import uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _check(ktau, X, path, count_bits):
    m, n = X.shape
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    res = ktau.allpairs(Xd, count_bits=count_bits, options={"path": path, "statistic": 1})
    torch.cuda.synchronize()
    ktau.ktau_device_status()
    got = {k: v.cpu().numpy() for k, v in res.items() if isinstance(v, torch.Tensor)}
    res["ranked"].free()
    ref = oracle_full(X)
    assert np.array_equal(got["S"].astype(np.int64), ref["S"])
    ta64 = np.array([oracle.tau_a(s, n) for s in ref["S"]], dtype=np.float64)
    ta32 = np.array([oracle.tau_a32(s, n) for s in ref["S"]], dtype=np.float32)
    assert np.array_equal(got["tau64"].view(np.int64), ta64.view(np.int64))
    assert np.array_equal(got["tau32"].view(np.int32), ta32.view(np.int32))


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("count_bits", [32, 64])
def test_tau_a_both_paths(ktau, path, count_bits):
    X = uniform_ties(150, 200, tie_frac=0.3, seed=3)
    X[4] = 2.0  # constant variable: tau-a is still defined (S = 0)
    _check(ktau, X, path, count_bits)


def test_tau_a_long_vectors(ktau):
    """n = 6000: n_0 = 17,997,000 > 2^24, so the FP32 value goes through the FP64 quotient and
    its midpoint check."""
    X = uniform_ties(12, 6000, tie_frac=0.2, seed=4)
    X[1] = X[0]
    X[2] = -X[0]
    _check(ktau, X, 1, 64)


def test_tau_a_rejected_by_query_and_batch(ktau):
    X = uniform_ties(20, 50, seed=5)
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    S = torch.empty((20, 20), dtype=torch.int32, device="cuda")
    with pytest.raises(ktau.KtauError):
        ktau.ktau_query(R, R, None, S, None, 32, 0, None, None, {"statistic": 1})
    R.free()
    o = torch.empty(190, dtype=torch.float32, device="cuda")
    with pytest.raises(ktau.KtauError):
        ktau.Batch([ktau.batch_desc(Xd, None, o, None, None, 32, 0)], options={"statistic": 1},
                   keepalive=[Xd])
