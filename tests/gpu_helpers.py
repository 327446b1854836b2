"""Shared helpers for the GPU parity tests (comparison against the CPU oracle)."""
import os

import numpy as np

import oracle

TAU_RTOL = 1e-12  # FP64 tau-b tolerance (both sides evaluate the same IEEE expression)


def pair_coords(m, ps):
    """(i, j) of packed strict-upper indices (oracle bijection on the (m-1)-triangle)."""
    out = []
    for p in ps:
        i, jm1 = oracle.job_coord(m - 1, int(p))
        out.append((i, jm1 + 1))
    return out


def oracle_sampled(X, ps):
    """Knight counts and tau-b of the pairs with the given packed indices."""
    m, n = X.shape
    Xd = np.asarray(X, dtype=np.float64)
    S, n3, tau = [], [], []
    for i, j in pair_coords(m, ps):
        c = oracle.pair_counts(Xd[i], Xd[j], "knight")
        S.append(c["S"])
        n3.append(c["n3"])
        tau.append(oracle.tau_b(c["S"], c["n1"], c["n2"], n))
    return np.array(S, np.int64), np.array(n3, np.int64), np.array(tau, np.float64)


def oracle_full(X, p_begin=0, p_end=None):
    return oracle.allpairs(np.asarray(X, dtype=np.float64), method="knight",
                           threads=os.cpu_count() or 1, p_begin=p_begin, p_end=p_end)


def assert_tau64(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    nan_g, nan_r = np.isnan(got), np.isnan(ref)
    assert np.array_equal(nan_g, nan_r), "NaN positions differ"
    ok = ~nan_r
    err = np.abs(got[ok] - ref[ok])
    bad = err > TAU_RTOL * np.abs(ref[ok])
    assert not bad.any(), f"{bad.sum()} tau64 values beyond 1e-12 relative; worst {err.max()}"


def assert_tau32(got, ref):
    got = np.asarray(got, np.float32)
    r32 = np.asarray(ref, np.float64).astype(np.float32)
    nan_g, nan_r = np.isnan(got), np.isnan(r32)
    assert np.array_equal(nan_g, nan_r), "NaN positions differ"
    ok = ~nan_r
    # FP32 output = round-to-nearest of the FP64 value: equal to rounding the oracle's FP64.
    assert np.array_equal(got[ok], r32[ok]), "tau32 differs from RN(oracle tau64)"
