"""CPU oracle for exact all-pairs Kendall tau-b (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package. It shares no code with the CUDA library and the
product path never routes through it.

The arithmetic lives in ``ktau_oracle.c`` (plain C, FP64 inputs, int64 counts), written from
arXiv 1704.03767:

* ``pair_counts(u, v, method="definition")`` -- Sec. 1 / Table 1 definition, O(n^2), sign
  form of Algorithm 1 extended with the tie counts n_1, n_2, n_3.
* ``pair_counts(u, v, method="knight")`` -- Sec. 3.2 Steps 1-5 with Algorithm 2.
* ``tau_b`` -- Eq. 3.
* ``tau_a`` / ``tau_a32`` / ``rn32`` -- tau-a of Sec. 2 ((n_c - n_d) / n_0) in FP64, and a
  quotient of integers rounded exactly to FP32 (round to nearest, ties to even).
* ``job_id`` / ``job_coord`` / ``job_coord_formula`` -- Eq. 4-10 (diagonal included).
* ``rank`` -- the per-variable rank transform of Sec. 3.
* ``allpairs`` -- Sec. 4.2-4.3 tiled walk of the upper triangle, static thread ranges.
* ``rect`` / ``query_topk`` -- query search of Sec. 1 with exact ordering by |tau|.
* ``permutation_exceed`` -- permutation test of every pair: exceedances |S(x_i, x_j o sigma)| >=
  |S(x_i, x_j)| over caller-drawn permutations sigma.

Parity pins for every function are in ``tests/test_oracle_pins.py`` and
``tests/test_bijection.py``; no function is "parity unpinned".
"""
from .oracle import (  # noqa: F401
    allpairs,
    build,
    job_coord,
    job_coord_formula,
    job_id,
    lib_path,
    pair_counts,
    permutation_exceed,
    query_topk,
    rank,
    rect,
    rn32,
    tau_a,
    tau_a32,
    tau_b,
    topk_order,
)
