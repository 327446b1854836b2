"""Autotuner: measures, on the GPU at hand, how long each pairwise path takes per pair and picks,
per sample count n and tie density, the fastest exact path and merge-path mapping.

    python -m paper_1704_03767_gb300.autotune            # measure and write tuning/<gpu>.json
    from paper_1704_03767_gb300 import autotune
    table = autotune.load()                              # table of the current GPU (or None)
    autotune.choose(table, n, tie_frac)                  # -> options dict for ktau_allpairs
    autotune.batch_paths(table, matrices)                # -> per-dataset path for ktau_batch

Candidates per (n, tie density): the merge path with one warp per pair (tile side 32 or 8) and
with one CTA per pair (n > 256), the bit-parallel dominance count (n <= 256), and the sign
contraction (n <= 2048 measured; it applies up to n = 5792) with block-scaled FP4 operands (the
default) or FP8 operands. Times come
from the library's own kernel trace (CUDA events around each launch), best of a few repetitions,
operands and masks already built (the first call builds them).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import binding as kb

TUNING_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning")
N_GRID = [20, 32, 64, 100, 128, 160, 200, 256, 384, 512, 768, 1024, 1500, 2000]
TIE_GRID = [0.05, 0.30]


def _gpu_key() -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "".join(c if c.isalnum() else "_" for c in name)


def _matrix(m: int, n: int, tie_frac: float, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    x = g.random((m, n))
    k = max(1, int(round(tie_frac * n)))
    dst = np.argpartition(g.random((m, n)), k - 1, axis=1)[:, :k] if k < n else \
        np.tile(np.arange(n), (m, 1))
    src = g.integers(0, n, size=(m, k))
    rows = np.arange(m)[:, None]
    x[rows, dst] = x[rows, src]
    return x.astype(np.float32)


def _time_pairs(R, P, opts, reps=3) -> float:
    """Best per-launch kernel time (ms) of ktau_allpairs over all pairs with these options."""
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    t32 = torch.empty(P, dtype=torch.float32, device="cuda")
    n3 = torch.empty(P, dtype=torch.int32, device="cuda")
    kb.ktau_allpairs(R, 0, P, None, t32, S, n3, 32, opts)  # warm-up (builds operands once)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        kb.ktau_trace_collect()
        kb.ktau_trace_enable(True)
        kb.ktau_allpairs(R, 0, P, None, t32, S, n3, 32, opts)
        kb.ktau_trace_enable(False)
        tr = kb.ktau_trace_collect()
        best = min(best, sum(ms for _, ms in tr))
    return best


def measure(n_grid=N_GRID, tie_grid=TIE_GRID, target_pairs=2_000_000, verbose=True) -> dict:
    entries = []
    for tie in tie_grid:
        for n in n_grid:
            m = int((2 * target_pairs) ** 0.5) + 1
            if n >= 1024:
                m = min(m, 1400)
            X = torch.from_numpy(_matrix(m, n, tie, seed=n)).cuda()
            R = kb.ktau_rank_prepare(X)
            P = m * (m - 1) // 2
            cands = {"merge_warp_q32": {"path": 1, "mapping": 1, "tile_q": 32},
                     "merge_warp_q8": {"path": 1, "mapping": 1, "tile_q": 8}}
            if n > 256:
                cands["merge_cta_q4"] = {"path": 1, "mapping": 2, "tile_q": 4}
            if n <= kb.KTAU_BITS_MAX_N:
                cands["bits"] = {"path": kb.KTAU_PATH_BITS}
            if n <= 2048:
                cands["signgemm"] = {"path": 2}
                cands["signgemm_fp8"] = {"path": 2, "operand_bits": 8}
            times = {}
            for name, o in cands.items():
                try:
                    times[name] = _time_pairs(R, P, o) * 1e6 / P  # ns per pair
                except kb.KtauError as e:
                    times[name] = None
                    if verbose:
                        print(f"  n={n} {name}: {e}")
            R.free()
            ok = {k: v for k, v in times.items() if v is not None}
            best = min(ok, key=ok.get)
            entries.append({"n": n, "tie_frac": tie, "m": m, "ns_per_pair": times, "best": best,
                            "options": cands[best]})
            if verbose:
                print(f"tie={tie:.2f} n={n:5d} m={m}: " + ", ".join(
                    f"{k}={v:.4f}" for k, v in ok.items()) + f" -> {best}", flush=True)
    return {"gpu": torch.cuda.get_device_name(), "sm_count":
            torch.cuda.get_device_properties(0).multi_processor_count, "entries": entries}


def save(table: dict, path: str | None = None) -> str:
    os.makedirs(TUNING_DIR, exist_ok=True)
    path = path or os.path.join(TUNING_DIR, _gpu_key() + ".json")
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    return path


def load(path: str | None = None):
    path = path or os.path.join(TUNING_DIR, _gpu_key() + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def choose(table, n: int, tie_frac: float = 0.05) -> dict:
    """Options of the fastest measured candidate at the nearest grid point (log n), or the
    library's built-in choice (path AUTO) without a table."""
    if not table:
        return {"path": kb.KTAU_PATH_AUTO}
    ents = table["entries"]
    ties = sorted({e["tie_frac"] for e in ents}, key=lambda t: abs(t - tie_frac))
    cand = [e for e in ents if e["tie_frac"] == ties[0]]
    e = min(cand, key=lambda e: abs(np.log(e["n"]) - np.log(n)))
    opts = dict(e["options"])
    if opts.get("path") == kb.KTAU_PATH_SIGNGEMM and n > 5792:
        opts = {"path": kb.KTAU_PATH_MERGE, "mapping": 2}
    return opts


def tie_fraction(X: np.ndarray, rows: int = 32) -> float:
    """Share of entries that repeat an earlier value of their row, on a few sampled rows."""
    Xs = np.asarray(X)[: max(1, min(rows, X.shape[0]))]
    reps = [1.0 - len(np.unique(r)) / len(r) for r in Xs]
    return float(np.mean(reps))


# Candidates the batched form can run (it has no bit-parallel path and one operand type per call).
_BATCHABLE = ("merge_warp_q32", "merge_warp_q8", "merge_cta_q4", "signgemm")


def choose_batch(table, n: int, tie_frac: float = 0.05) -> dict:
    """Fastest batchable candidate at the nearest grid point: {"path", "mapping"}."""
    if not table:
        return {"path": kb.KTAU_PATH_AUTO, "mapping": 0}
    ents = table["entries"]
    ties = sorted({e["tie_frac"] for e in ents}, key=lambda t: abs(t - tie_frac))
    e = min((e for e in ents if e["tie_frac"] == ties[0]),
            key=lambda e: abs(np.log(e["n"]) - np.log(n)))
    times = {k: v for k, v in e["ns_per_pair"].items() if k in _BATCHABLE and v is not None}
    best = min(times, key=times.get)
    if best == "signgemm" and n <= 3000:  # the batched contraction's n_3 takes n <= 3000
        return {"path": kb.KTAU_PATH_SIGNGEMM, "mapping": 0}
    if best == "signgemm":
        best = "merge_cta_q4"
    return {"path": kb.KTAU_PATH_MERGE, "mapping": 2 if best == "merge_cta_q4" else 1}


def batch_paths(table, matrices) -> list:
    """Per-dataset path (ktau_path) for the batched form."""
    return [choose_batch(table, X.shape[1], tie_fraction(X))["path"] for X in matrices]


def batch_plans(table, matrices) -> list:
    """Per-dataset (path, merge mapping) for the batched form's descriptors."""
    return [choose_batch(table, X.shape[1], tie_fraction(X)) for X in matrices]


if __name__ == "__main__":
    import sys

    t = measure()
    print(save(t, sys.argv[1] if len(sys.argv) > 1 else None))
