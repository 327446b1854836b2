"""Batched form: many uneven datasets in one persistent launch per kernel family, optionally
replayed from a CUDA graph. Every dataset must match the oracle exactly and be bit-identical to
the plain per-dataset launch (both store through the same epilogue)."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_tau32, assert_tau64, oracle_full, oracle_sampled
from synthetic import batched_shapes, batched_uneven, uniform_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ktau():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as k

    k.load()
    return k


def _make(ktau, mats, count_bits=64, paths=None, options=None):
    descs, outs, keep = [], [], []
    for i, X in enumerate(mats):
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        m = X.shape[0]
        P = m * (m - 1) // 2
        cdt = torch.int64 if count_bits == 64 else torch.int32
        o = {"tau64": torch.full((P,), -7.0, dtype=torch.float64, device="cuda"),
             "tau32": torch.full((P,), -7.0, dtype=torch.float32, device="cuda"),
             "S": torch.full((P,), -99, dtype=cdt, device="cuda"),
             "n3": torch.full((P,), -99, dtype=cdt, device="cuda")}
        descs.append(ktau.batch_desc(Xd, o["tau64"], o["tau32"], o["S"], o["n3"], count_bits,
                                     0 if paths is None else paths[i]))
        outs.append(o)
        keep.append(Xd)
    B = ktau.Batch(descs, options=options, keepalive=keep)
    return B, outs


def _np(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("mode,bits", [("auto", 0), ("merge", 0), ("signgemm", 0),
                                       ("signgemm", 4), ("signgemm", 16)])
def test_small_batch_matches_oracle(ktau, mode, bits):
    mats = batched_uneven(count=24, m_range=(16, 150), n_range=(20, 300), seed0=100)
    mats[3][5] = 1.0  # a constant variable
    if mode != "signgemm":  # the batched contraction counts n_3 for n <= 3000 only
        mats.append(uniform_ties(40, 3100, tie_frac=0.1, seed=5))  # long vectors: merge path
    paths = None if mode == "auto" else [1 if mode == "merge" else 2] * len(mats)
    B, outs = _make(ktau, mats, 64, paths, {"operand_bits": bits} if bits else None)
    nm, ns = B.paths()
    if mode == "merge":
        assert ns == 0
    if mode == "signgemm":
        assert nm == 0
    if mode == "auto":
        assert nm > 0 and ns > 0
    s = torch.cuda.Stream()
    B.run(s)
    B.check(s)
    for X, o in zip(mats, outs):
        got = _np(o)
        ref = oracle_full(X)
        assert np.array_equal(got["S"], ref["S"])
        assert np.array_equal(got["n3"], ref["n3"])
        assert_tau64(got["tau64"], ref["tau"])
        assert_tau32(got["tau32"], ref["tau"])
    B.free()


def test_graph_replay_and_plain_launch_identity(ktau):
    mats = batched_uneven(count=30, m_range=(16, 300), n_range=(20, 700), seed0=7)
    B, outs = _make(ktau, mats, 32)
    s = torch.cuda.Stream()
    B.graph_launch(s)
    B.check(s)
    first = [_np(o) for o in outs]
    for o in outs:
        for t in o.values():
            t.fill_(-5)
    B.graph_launch(s)  # replay
    B.check(s)
    for X, o, f in zip(mats, outs, first):
        g = _np(o)
        for k in g:
            assert np.array_equal(g[k].view(np.int32 if g[k].itemsize == 4 else np.int64),
                                  f[k].view(np.int32 if f[k].itemsize == 4 else np.int64))
        # plain launch of the same dataset: bit-identical outputs
        p = ktau.allpairs(torch.from_numpy(X).cuda(), count_bits=32)
        torch.cuda.synchronize()
        for k in ("tau64", "tau32", "S", "n3"):
            a = p[k].cpu().numpy()
            assert np.array_equal(a.view(np.int32 if a.itemsize == 4 else np.int64),
                                  g[k].view(np.int32 if a.itemsize == 4 else np.int64)), k
        p["ranked"].free()
    B.free()


def test_nan_reported(ktau):
    mats = [uniform_ties(20, 30, seed=1), uniform_ties(25, 40, seed=2)]
    mats[1][3, 4] = np.nan
    B, outs = _make(ktau, mats, 32)
    s = torch.cuda.Stream()
    B.run(s)
    with pytest.raises(ktau.KtauError) as ei:
        B.check(s)
    assert ei.value.status == 2
    B.free()


def test_invalid_descriptors(ktau):
    X = torch.zeros((1, 10), device="cuda")
    with pytest.raises(ktau.KtauError):
        ktau.Batch([ktau.batch_desc(X)])


def test_thousand_uneven_datasets_sampled(ktau):
    """The batched workload: 1000 matrices, m log-uniform in [16, 1024], n in [20, 2000]."""
    mats = batched_uneven(count=1000, seed0=0)
    assert [x.shape for x in mats[:5]] == batched_shapes(5)
    B, outs = _make(ktau, mats, 32)
    s = torch.cuda.Stream()
    B.graph_launch(s)
    B.check(s)
    g = np.random.default_rng(0)
    for i in g.choice(len(mats), 25, replace=False):
        X, o = mats[i], outs[i]
        m = X.shape[0]
        P = m * (m - 1) // 2
        ps = np.unique(np.concatenate([g.integers(0, P, 40), [0, P - 1]]))
        rS, rn3, rtau = oracle_sampled(X, ps)
        idx = torch.from_numpy(ps).cuda()
        assert np.array_equal(o["S"][idx].cpu().numpy().astype(np.int64), rS)
        assert np.array_equal(o["n3"][idx].cpu().numpy().astype(np.int64), rn3)
        assert_tau64(o["tau64"][idx].cpu().numpy(), rtau)
        assert_tau32(o["tau32"][idx].cpu().numpy(), rtau)
    B.free()


def _bits(a):
    return a.view(np.int32 if a.itemsize == 4 else np.int64)


def _descs_like(ktau, mats, count_bits=32, paths=None):
    """Fresh outputs and descriptors for the one-call form (same datasets as a plan)."""
    descs, outs, keep = [], [], []
    for i, X in enumerate(mats):
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        m = X.shape[0]
        P = m * (m - 1) // 2
        cdt = torch.int64 if count_bits == 64 else torch.int32
        o = {"tau64": torch.full((P,), -3.0, dtype=torch.float64, device="cuda"),
             "tau32": torch.full((P,), -3.0, dtype=torch.float32, device="cuda"),
             "S": torch.full((P,), -9, dtype=cdt, device="cuda"),
             "n3": torch.full((P,), -9, dtype=cdt, device="cuda")}
        descs.append(ktau.batch_desc(Xd, o["tau64"], o["tau32"], o["S"], o["n3"], count_bits,
                                     0 if paths is None else paths[i]))
        outs.append(o)
        keep.append(Xd)
    return descs, outs, keep


def _workspace(nbytes):
    # 256-byte aligned view into a byte tensor (torch's allocator aligns to 512 bytes anyway)
    return torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")[:nbytes]


@pytest.mark.parametrize("paths", [None, "merge"])
def test_batched_call_matches_plan(ktau, paths):
    """ktau_allpairs_batched (scratch in the caller's workspace, one stream) gives the plan's
    outputs bit for bit, twice in a row on the same workspace, and a graph captured around it
    replays the same outputs."""
    mats = batched_uneven(count=40, m_range=(16, 260), n_range=(20, 1400), seed0=300)
    mats[2][4] = 2.0  # constant variable
    pth = None if paths is None else [1] * len(mats)
    B, ref_outs = _make(ktau, mats, 32, pth)
    s = torch.cuda.Stream()
    B.run(s)
    B.check(s)
    ref = [_np(o) for o in ref_outs]
    B.free()
    descs, outs, keep = _descs_like(ktau, mats, 32, pth)
    nbytes = ktau.ktau_workspace_size(descs)
    ws = _workspace(nbytes)
    assert ws.data_ptr() % 256 == 0
    flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    for rep in range(2):
        for o in outs:
            for t in o.values():
                t.fill_(-4)
        ktau.ktau_allpairs_batched(descs, ws, flag, stream=s)
        s.synchronize()
        assert int(flag.item()) == 0
        for o, r in zip(outs, ref):
            g = _np(o)
            for k in g:
                assert np.array_equal(_bits(g[k]), _bits(r[k])), (rep, k)
    # capture the call into a graph and replay it
    for o in outs:
        for t in o.values():
            t.fill_(-4)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ktau.ktau_allpairs_batched(descs, ws, flag, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        got = _np(o)
        for k in got:
            assert np.array_equal(_bits(got[k]), _bits(r[k])), ("graph", k)
    del g
    ktau.ktau_device_status(s)


def test_batched_call_nan_and_small_workspace(ktau):
    mats = [uniform_ties(20, 30, seed=1), uniform_ties(25, 40, seed=2)]
    mats[1][3, 4] = np.nan
    descs, outs, keep = _descs_like(ktau, mats)
    nbytes = ktau.ktau_workspace_size(descs)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    ktau.ktau_allpairs_batched(descs, _workspace(nbytes), flag)
    torch.cuda.synchronize()
    assert int(flag.item()) != 0
    with pytest.raises(ktau.KtauError) as ei:
        ktau.ktau_allpairs_batched(descs, _workspace(nbytes - 256), flag)
    assert ei.value.status == 1 and "workspace" in ei.value.message
