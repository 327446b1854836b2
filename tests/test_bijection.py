"""Pins of the job-id <-> (y, x) bijection (Sec. 4.1, Eq. 4-10) by brute-force enumeration.

The numbering policy of Sec. 4.1 is: jobs of the upper triangle (diagonal included) numbered
left to right, top to bottom. Enumerating the cells in that order and counting gives every
id without using Eq. 4-10, so the enumeration pins both directions of the oracle.
"""
import numpy as np

import pytest


def test_roundtrip_exhaustive(oracle_mod):
    for m in list(range(1, 90)) + [127, 128, 129, 200]:
        J = 0
        for y in range(m):
            for x in range(y, m):
                assert oracle_mod.job_id(m, y, x) == J
                assert oracle_mod.job_coord(m, J) == (y, x)
                J += 1


def test_paper_formula_exhaustive(oracle_mod):
    """Eq. 9-10 evaluated in FP64 without any integer correction, small m."""
    bad = 0
    for m in range(1, 130):
        J = 0
        for y in range(m):
            for x in range(y, m):
                bad += oracle_mod.job_coord_formula(m, J) != (y, x)
                J += 1
    assert bad == 0


@pytest.mark.parametrize("m", [1000, 16383, 16384, 65536, 1 << 20, (1 << 22) + 3])
def test_row_boundaries_large(oracle_mod, m):
    # first id of each row = running sum of the row lengths m, m-1, ... (enumeration, not Eq. 5)
    lengths = m - np.arange(m, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    g = np.random.default_rng(m)
    ys = np.unique(np.concatenate([np.arange(min(m, 64)), np.arange(max(0, m - 64), m),
                                   g.integers(0, m, 400)]))
    for y in ys:
        y = int(y)
        first = int(starts[y])
        last = first + m - y - 1
        assert oracle_mod.job_coord(m, first) == (y, y)
        assert oracle_mod.job_coord(m, last) == (y, m - 1)
        assert oracle_mod.job_id(m, y, y) == first


def test_strict_upper_packed_index(oracle_mod):
    """The ABI's packed strict-upper index p(i, j) equals the Eq. 4 id on the (m-1)-triangle
    at (i, j-1); enumeration of pairs i<j in row-major order pins it."""
    for m in (2, 3, 7, 64, 65):
        p = 0
        for i in range(m):
            for j in range(i + 1, m):
                assert oracle_mod.job_id(m - 1, i, j - 1) == p
                assert oracle_mod.job_coord(m - 1, p) == (i, j - 1)
                p += 1
