"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-worked counts (tests/golden/hand_worked.txt, counted pair by pair from Sec. 1 / Table 1)
* scipy.stats.kendalltau (tau-b), an independent library implementation of Eq. 3
* identities: tau(u,u) = 1 and tau(u, reverse u) = -1 without ties; symmetry (Sec. 1: the
  computation is commutable); tau-a = tau-b without ties (Sec. 1, after Eq. 3)
* brute force: the O(n^2) definition and the O(n log n) Knight counter (Sec. 3.2) agree on
  every pair of vectors over small alphabets (exhaustive)
* the Step 5 identity n_c - n_d = n_0 - n_1 - n_2 + n_3 - 2 n_d on definition-level counts
* rank transform against numpy's stable argsort and np.unique
"""
import itertools
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        u, v, c, t = [p.strip() for p in line.split("|")]
        rows.append(
            (
                np.array([float(x) for x in u.split()]),
                np.array([float(x) for x in v.split()]),
                [int(x) for x in c.split()],
                float(t),
            )
        )
    return rows


@pytest.mark.parametrize("method", ["definition", "knight"])
def test_hand_worked(oracle_mod, method):
    rows = _golden_rows()
    assert len(rows) >= 8
    for u, v, (nc, nd, n1, n2, n3, S), tau in rows:
        c = oracle_mod.pair_counts(u, v, method)
        assert (c["nc"], c["nd"], c["n1"], c["n2"], c["n3"], c["S"]) == (nc, nd, n1, n2, n3, S), (
            u, v, c)
        t = oracle_mod.tau_b(c["S"], c["n1"], c["n2"], len(u))
        if math.isnan(tau):
            assert math.isnan(t)
        else:
            assert abs(t - tau) <= 1e-15 * max(1.0, abs(tau)), (t, tau)


def test_scipy_tau_b(oracle_mod):
    stats = pytest.importorskip("scipy.stats")
    g = np.random.default_rng(11)
    for trial in range(300):
        n = int(g.integers(2, 60))
        levels = int(g.integers(2, 12)) if trial % 2 else 1000
        u = g.integers(0, levels, n).astype(float)
        v = g.integers(0, levels, n).astype(float)
        if trial % 5 == 0:
            v = u + g.integers(-1, 2, n)
        c = oracle_mod.pair_counts(u, v, "knight")
        t = oracle_mod.tau_b(c["S"], c["n1"], c["n2"], n)
        ref = stats.kendalltau(u, v).statistic
        if math.isnan(ref):
            assert math.isnan(t)
        else:
            assert abs(t - ref) <= 1e-12 * max(1.0, abs(ref)), (u, v, t, ref)


def test_identities(oracle_mod):
    g = np.random.default_rng(5)
    for n in (2, 3, 17, 128, 257):
        u = g.permutation(n).astype(float) + 0.5
        for method in ("definition", "knight"):
            c = oracle_mod.pair_counts(u, u, method)
            assert c["S"] == n * (n - 1) // 2 and c["nd"] == 0
            assert oracle_mod.tau_b(c["S"], c["n1"], c["n2"], n) == 1.0
            # reversing the order of the values (v = -u) gives the exact anti-order
            c = oracle_mod.pair_counts(u, -u, method)
            assert c["S"] == -(n * (n - 1) // 2) and c["nc"] == 0
            assert oracle_mod.tau_b(c["S"], c["n1"], c["n2"], n) == -1.0
        us = np.sort(u)
        for method in ("definition", "knight"):
            c = oracle_mod.pair_counts(us, us[::-1].copy(), method)
            assert c["S"] == -(n * (n - 1) // 2) and c["nc"] == 0
            assert oracle_mod.tau_b(c["S"], c["n1"], c["n2"], n) == -1.0


def test_symmetry_and_tau_a(oracle_mod):
    g = np.random.default_rng(7)
    for trial in range(200):
        n = int(g.integers(2, 80))
        u = g.integers(0, 6 if trial % 2 else 10**6, n).astype(float)
        v = g.integers(0, 6 if trial % 3 else 10**6, n).astype(float)
        a = oracle_mod.pair_counts(u, v, "knight")
        b = oracle_mod.pair_counts(v, u, "knight")
        assert (a["S"], a["n3"], a["n1"], a["n2"]) == (b["S"], b["n3"], b["n2"], b["n1"])
        ta = oracle_mod.tau_b(a["S"], a["n1"], a["n2"], n)
        tb = oracle_mod.tau_b(b["S"], b["n1"], b["n2"], n)
        assert (math.isnan(ta) and math.isnan(tb)) or ta == tb
        if a["n1"] == 0 and a["n2"] == 0:
            n0 = n * (n - 1) // 2
            assert abs(ta - a["S"] / n0) <= 1e-15
            assert a["nc"] + a["nd"] == n0


def test_brute_force_exhaustive(oracle_mod):
    """Definition and Knight agree on every (u, v) over a 3-letter alphabet, n = 1..5."""
    for n in range(1, 6):
        vecs = [np.array(t, float) for t in itertools.product(range(3), repeat=n)]
        for u in vecs:
            for v in vecs[:: max(1, len(vecs) // 40)]:
                a = oracle_mod.pair_counts(u, v, "definition")
                b = oracle_mod.pair_counts(u, v, "knight")
                assert a == b, (u, v, a, b)


def test_brute_force_random(oracle_mod):
    g = np.random.default_rng(3)
    for trial in range(300):
        n = int(g.integers(2, 300))
        lv = [2, 3, 8, 64, 10**9][trial % 5]
        u = g.integers(0, lv, n).astype(float)
        v = g.integers(0, [2, 5, 64, 10**9][trial % 4], n).astype(float)
        a = oracle_mod.pair_counts(u, v, "definition")
        b = oracle_mod.pair_counts(u, v, "knight")
        assert a == b
        n0 = n * (n - 1) // 2
        # Step 5 (Sec. 3.2) on definition-level counts
        assert a["nc"] - a["nd"] == n0 - a["n1"] - a["n2"] + a["n3"] - 2 * a["nd"]


def test_rank_transform(oracle_mod):
    g = np.random.default_rng(9)
    for trial in range(100):
        n = int(g.integers(1, 500))
        x = g.integers(0, [3, 50, 10**9][trial % 3], n).astype(float)
        if trial % 7 == 0:
            x[g.integers(0, n)] = -0.0
            x[g.integers(0, n)] = 0.0
        perm, rk, T = oracle_mod.rank(x)
        assert np.array_equal(perm, np.argsort(x, kind="stable"))
        uniq, inv, cnt = np.unique(x, return_inverse=True, return_counts=True)
        assert np.array_equal(rk, inv)
        assert T == int((cnt * (cnt - 1) // 2).sum())


def test_allpairs_matches_pairs(oracle_mod):
    g = np.random.default_rng(1)
    m, n = 21, 33
    X = g.integers(0, 7, (m, n)).astype(float)
    ref = []
    for i in range(m):
        for j in range(i + 1, m):
            ref.append(oracle_mod.pair_counts(X[i], X[j], "definition"))
    P = m * (m - 1) // 2
    for method, q, threads in (("knight", 8, 1), ("knight", 3, 4), ("definition", 5, 3)):
        out = oracle_mod.allpairs(X, method=method, q=q, threads=threads)
        assert [int(s) for s in out["S"]] == [r["S"] for r in ref]
        assert [int(s) for s in out["n3"]] == [r["n3"] for r in ref]
    # sub-ranges (Sec. 4.3.1 passes) concatenate to the full result
    full = oracle_mod.allpairs(X)
    cuts = [0, 1, 50, 51, 199, P]
    parts = [oracle_mod.allpairs(X, p_begin=a, p_end=b)["S"] for a, b in zip(cuts, cuts[1:])]
    assert np.array_equal(np.concatenate(parts), full["S"])


def test_topk_order(oracle_mod):
    # exact ordering by |tau| with index tie-break, NaN last
    S = [3, -3, 0, 5, 3, -5]
    Dv = [10, 10, 10, 0, 9, 25]
    # |tau|^2 * Du = S^2/Dv: 0.9, 0.9, 0, nan, 1.0, 1.0
    assert oracle_mod.topk_order(S, 7, Dv, 6) == [4, 5, 0, 1, 2, 3]
    assert oracle_mod.topk_order(S, 0, Dv, 3) == [0, 1, 2]


# ---------------------------------------------------------------------------------------------
# tau-a (Sec. 2: (n_c - n_d) / n_0) and the exact FP32 rounding of a quotient
# ---------------------------------------------------------------------------------------------
def test_rn32_matches_ieee_float32_division(oracle_mod):
    """Where both operands are exact in FP32, IEEE single division (numpy) is correctly rounded,
    so it must agree with the exact rounding bit for bit."""
    g = np.random.default_rng(7)
    nums = g.integers(-(1 << 24) + 1, 1 << 24, 20000)
    dens = g.integers(1, 1 << 24, 20000)
    for a, b in zip(nums, dens):
        ref = np.float32(a) / np.float32(b)
        got = oracle_mod.rn32(int(a), int(b))
        assert got.view(np.uint32) == ref.view(np.uint32), (a, b)


def test_rn32_ties_and_nearest_property(oracle_mod):
    from fractions import Fraction

    # exact midpoints: ties to the even significand
    assert oracle_mod.rn32((1 << 24) + 1, 1 << 25) == np.float32(0.5)
    assert oracle_mod.rn32((1 << 24) + 3, 1 << 25) == np.float32(0.5 + 2.0 ** -23)
    assert oracle_mod.rn32(-((1 << 24) + 1), 1 << 25) == np.float32(-0.5)
    # nearest-value property in exact arithmetic, with denominators beyond FP32's exact range
    g = np.random.default_rng(8)
    for _ in range(3000):
        den = int(g.integers(1 << 24, 1 << 30))
        num = int(g.integers(-den, den + 1))
        if num == 0:
            continue
        f = oracle_mod.rn32(num, den)
        x = Fraction(num, den)
        fx = Fraction(float(f))
        for nb in (np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))):
            d_nb, d_f = abs(x - Fraction(float(nb))), abs(x - fx)
            assert d_f < d_nb or (d_f == d_nb and (f.view(np.uint32) & 1) == 0)


def test_tau_a_definition(oracle_mod):
    """tau-a against the definition on tiny inputs, and tau-a = tau-b without ties."""
    g = np.random.default_rng(9)
    for _ in range(200):
        n = int(g.integers(2, 9))
        u, v = g.integers(0, 4, n), g.integers(0, 4, n)
        nc = sum(1 for a in range(n) for b in range(a + 1, n) if (u[a] - u[b]) * (v[a] - v[b]) > 0)
        nd = sum(1 for a in range(n) for b in range(a + 1, n) if (u[a] - u[b]) * (v[a] - v[b]) < 0)
        c = oracle_mod.pair_counts(u.astype(float), v.astype(float))
        assert oracle_mod.tau_a(c["S"], n) == (nc - nd) / (n * (n - 1) / 2)
    u = g.permutation(30).astype(float)
    v = g.permutation(30).astype(float)
    c = oracle_mod.pair_counts(u, v)
    assert abs(oracle_mod.tau_a(c["S"], 30) - oracle_mod.tau_b(c["S"], 0, 0, 30)) < 1e-15


# ---------------------------------------------------------------------------------------------
# Permutation test of every pair
# ---------------------------------------------------------------------------------------------
def _mahonian(n):
    """Number of permutations of n items with k inversions, k = 0..n(n-1)/2 (standard recurrence)."""
    row = [1]
    for i in range(2, n + 1):
        new = [0] * (len(row) + i - 1)
        for k, c in enumerate(row):
            for j in range(i):
                new[k + j] += c
        row = new
    return row


def test_permutation_exceed_exact_null(oracle_mod):
    """Over all n! relabellings of a tie-free variable, S = n_0 - 2 * (inversions), so the number
    of permutations with |S_sigma| >= |S_obs| follows from the Mahonian distribution."""
    n = 6
    n0 = n * (n - 1) // 2
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.uint16)
    mah = _mahonian(n)
    g = np.random.default_rng(12)
    X = np.stack([g.permutation(n) for _ in range(4)]).astype(np.float64)
    exc = oracle_mod.permutation_exceed(X, perms)
    S_obs = oracle_mod.allpairs(X)["S"]
    for s_obs, e in zip(S_obs, exc):
        expect = sum(c for k, c in enumerate(mah) if abs(n0 - 2 * k) >= abs(s_obs))
        assert e == expect


def test_permutation_exceed_identity_and_ranges(oracle_mod):
    g = np.random.default_rng(13)
    X = np.round(g.random((9, 15)), 1)
    ident = np.tile(np.arange(15, dtype=np.uint16), (3, 1))
    assert np.all(oracle_mod.permutation_exceed(X, ident) == 3)
    perms = np.stack([g.permutation(15) for _ in range(5)]).astype(np.uint16)
    full = oracle_mod.permutation_exceed(X, perms)
    assert np.array_equal(oracle_mod.permutation_exceed(X, perms, 7, 30), full[7:30])
    assert np.all((full >= 0) & (full <= 5))


def test_allpairs_thread_slices(oracle_mod):
    """The requested range is cut into per-thread slices: any thread count and any sub-range give
    the single-thread result, including slices that start and end inside a tile row."""
    g = np.random.default_rng(21)
    m, n = 37, 19
    X = g.integers(0, 5, (m, n)).astype(float)
    P = m * (m - 1) // 2
    ref = oracle_mod.allpairs(X, threads=1)
    for threads in (2, 3, 7, 16, 40):
        for a, b in ((0, P), (0, 90), (13, 14), (200, 611), (P - 5, P)):
            out = oracle_mod.allpairs(X, q=4, threads=threads, p_begin=a, p_end=b)
            for k in ("S", "n3", "nd", "n1", "n2"):
                assert np.array_equal(out[k], ref[k][a:b]), (threads, a, b, k)


def _brute_topk(Q, D, k):
    """Independent top-k: per (query, row) the definition counter and Eq. 3, then a full sort on
    (tau is NaN, -|tau| as the exact rational S^2 / (D_u D_v), row index)."""
    from fractions import Fraction

    n = Q.shape[1]
    n0 = n * (n - 1) // 2
    idx, tau = [], []
    for q in Q:
        keyed = []
        for j, row in enumerate(D):
            c = pair_counts_def(q, row)
            du, dv = n0 - c["n1"], n0 - c["n2"]
            t = math.nan if du == 0 or dv == 0 else c["S"] / math.sqrt(du * dv)
            key = (1, Fraction(0)) if math.isnan(t) else (0, -Fraction(c["S"] ** 2, du * dv))
            keyed.append((key, j, t))
        keyed.sort(key=lambda e: (e[0], e[1]))
        idx.append([j for _, j, _ in keyed[:k]])
        tau.append([t for _, _, t in keyed[:k]])
    return idx, tau


def pair_counts_def(u, v):
    """Definition-level counts written out in Python (sign products over all sample pairs)."""
    u, v = [float(x) for x in u], [float(x) for x in v]
    nc = nd = n1 = n2 = 0
    n = len(u)
    for a in range(n):
        for b in range(a + 1, n):
            su = (u[a] > u[b]) - (u[a] < u[b])
            sv = (v[a] > v[b]) - (v[a] < v[b])
            nc += su * sv > 0
            nd += su * sv < 0
            n1 += su == 0
            n2 += sv == 0
    return {"S": nc - nd, "n1": n1, "n2": n2}


def test_query_topk_brute_force(oracle_mod):
    """query_topk against the brute-force order above. The database has rows with equal |tau|
    against the queries (duplicated and negated rows), a constant row (NaN, last) and tied values;
    one query is constant (every tau NaN: order by row index)."""
    g = np.random.default_rng(31)
    n = 9
    D = g.integers(0, 4, (14, n)).astype(float)
    D[3] = D[1]             # equal |tau| to row 1 for every query: index order decides
    D[5] = -D[1]            # |tau| equal to rows 1 and 3, sign flipped
    D[7] = 2.0              # constant row: NaN
    D[9] = g.permutation(n)  # no ties
    Q = g.integers(0, 5, (4, n)).astype(float)
    Q[2] = D[1]             # |tau| = 1 against rows 1, 3 and 5
    Q[3] = 1.5              # constant query
    for k in (1, 5, 14):
        r = oracle_mod.query_topk(Q, D, k)
        idx, tau = _brute_topk(Q, D, k)
        assert r["topk_idx"].tolist() == idx, k
        for got, want in zip(r["topk_tau"], tau):
            for a, b in zip(got, want):
                assert (math.isnan(a) and math.isnan(b)) or a == b
    r = oracle_mod.query_topk(Q, D, 14)
    assert r["topk_idx"][2][:3].tolist() == [1, 3, 5]
    assert r["topk_idx"][3].tolist() == list(range(14))
    assert 7 == r["topk_idx"][0][-1]
