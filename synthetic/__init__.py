"""Seeded synthetic inputs with the shapes of the paper's workloads.

This module holds no tau arithmetic: it only draws matrices. Both the CUDA path's tests and
the oracle read inputs from here, and nothing else is shared between them.

The paper measures on gene-expression matrices (genes x samples, about 17.9k x 310-353, from
the SEEK GPL570 collection; Sec. 5, Table 2), which are not available here. These generators
stand in for them with the same orientation (variables >> samples), log-normal expression
levels, shared latent structure, and quantisation ties.

Every generator uses ``numpy.random.Generator(PCG64(seed))`` and casts to the storage dtype
last. Optional size arguments shrink a workload to a parity-test size with the same recipe.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "uniform_ties",
    "gene_expression",
    "heavy_ties_ordinal",
    "batched_uneven",
    "batched_shapes",
    "query_batch_sizes",
    "poisson_arrivals",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_ties(m: int = 64, n: int = 200, tie_frac: float = 0.20, seed: int = 0) -> np.ndarray:
    """Uniform[0,1) values; a `tie_frac` share of entries, chosen without replacement, is
    rounded to 2 decimals so that ties appear. float32 [m, n]."""
    g = _rng(seed)
    x = g.random((m, n))
    k = int(round(tie_frac * m * n))
    flat = g.choice(m * n, size=k, replace=False)
    xf = x.reshape(-1)
    xf[flat] = np.round(xf[flat], 2)
    return x.astype(np.float32)


def gene_expression(m: int = 16384, n: int = 128, factors: int = 256, quant_frac: float = 0.10,
                    seed: int = 0) -> np.ndarray:
    """Gene-expression-shaped matrix, float32 [m, n].

    256 latent factors Z_k ~ N(0,1)^n; row i picks k_i and rho_i ~ U[0.3, 0.95] and draws
    y = rho_i Z_k + sqrt(1 - rho_i^2) eps; x = exp(2 + y) (log-normal, mu=2, sigma=1); then a
    random monotone transform, x**a (a ~ U[0.5, 2]) or log1p(c x) (c ~ U[0.1, 10]), 50/50;
    finally a `quant_frac` share of entries is quantised to round(10 x) / 10 (ties)."""
    g = _rng(seed)
    Z = g.standard_normal((factors, n))
    k = g.integers(0, factors, size=m)
    rho = g.uniform(0.3, 0.95, size=m)[:, None]
    eps = g.standard_normal((m, n))
    y = rho * Z[k] + np.sqrt(1.0 - rho * rho) * eps
    x = np.exp(2.0 + y)
    use_pow = g.random(m) < 0.5
    a = g.uniform(0.5, 2.0, size=m)[:, None]
    c = g.uniform(0.1, 10.0, size=m)[:, None]
    x = np.where(use_pow[:, None], x ** a, np.log1p(c * x))
    sel = g.random((m, n)) < quant_frac
    x = np.where(sel, np.round(x * 10.0) / 10.0, x)
    return x.astype(np.float32)


def heavy_ties_ordinal(m: int = 2048, n: int = 4096, levels: int = 64, tau_target: float = 0.3,
                       seed: int = 0) -> np.ndarray:
    """Long ordinal profiles with heavy ties, int32 [m, n] with values in 0..levels-1.

    A shared latent L ~ N(0,1)^n; the first half of the rows is rho L + sqrt(1-rho^2) eps with
    rho = sin(pi tau/2) (Greiner's relation gives Kendall tau ~ tau_target between such a row and
    L), the other half pure noise; value = floor(levels * Phi(y)) (uniform marginals)."""
    from scipy.special import ndtr

    g = _rng(seed)
    L = g.standard_normal(n)
    rho = math.sin(math.pi * tau_target / 2.0)
    eps = g.standard_normal((m, n))
    y = eps.copy()
    half = m // 2
    y[:half] = rho * L[None, :] + math.sqrt(1.0 - rho * rho) * eps[:half]
    v = np.floor(levels * ndtr(y))
    v = np.clip(v, 0, levels - 1)
    return v.astype(np.int32)


def batched_shapes(count: int = 1000, m_range=(16, 1024), n_range=(20, 2000), seed0: int = 0):
    """(m, n) of each dataset: log-uniform in the given ranges, dataset d seeded with seed0 + d."""
    shapes = []
    for d in range(count):
        g = _rng(seed0 + d)
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        shapes.append((m, n))
    return shapes


def batched_uneven(count: int = 1000, m_range=(16, 1024), n_range=(20, 2000), dup_frac=0.05,
                   seed0: int = 0):
    """List of `count` float32 matrices of uneven shape (see batched_shapes), uniform[0,1)
    values; in every row a `dup_frac` share of entries is overwritten with a copy of another
    entry of the same row (ties)."""
    out = []
    for d in range(count):
        g = _rng(seed0 + d)
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        x = g.random((m, n))
        k = max(1, int(round(dup_frac * n)))
        dst = np.argpartition(g.random((m, n)), k - 1, axis=1)[:, :k] if k < n else \
            np.tile(np.arange(n), (m, 1))
        src = g.integers(0, n, size=(m, k))
        rows = np.arange(m)[:, None]
        x[rows, dst] = x[rows, src]
        out.append(x.astype(np.float32))
    return out


def query_batch_sizes(count: int, max_batch: int = 512, seed: int = 2) -> list:
    """Batch sizes round(exp(U[0, ln max_batch])) (log-uniform in 1..max_batch)."""
    g = _rng(seed)
    return [max(1, int(round(math.exp(g.uniform(0.0, math.log(max_batch)))))) for _ in range(count)]


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 3) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    g = _rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def permutations(count: int, n: int, seed: int = 11) -> np.ndarray:
    """`count` uniformly random permutations of range(n) (PCG64, seeded), uint16 [count, n]: the
    sample relabellings a permutation test draws, generated here and passed to both sides."""
    g = _rng(seed)
    return np.stack([g.permutation(n) for _ in range(count)]).astype(np.uint16)
