"""ctypes wrapper around ``ktau_oracle.c`` (test infrastructure only; see package docstring)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ktau_oracle.c")
_LIB = os.path.join(_HERE, "libktau_oracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class _Counts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("nc", "nd", "n1", "n2", "n3")]


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no GPU code). Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.ko_pair_definition.argtypes = [_f64p, _f64p, ctypes.c_int64, ctypes.POINTER(_Counts)]
        lib.ko_pair_knight.argtypes = [_f64p, _f64p, ctypes.c_int64, ctypes.POINTER(_Counts)]
        lib.ko_pair_knight.restype = ctypes.c_int
        lib.ko_tau_b.argtypes = [ctypes.c_int64] * 4
        lib.ko_tau_b.restype = ctypes.c_double
        lib.ko_F.argtypes = [ctypes.c_int64, ctypes.c_int64]
        lib.ko_F.restype = ctypes.c_int64
        lib.ko_job_id.argtypes = [ctypes.c_int64] * 3
        lib.ko_job_id.restype = ctypes.c_int64
        for fn in (lib.ko_job_coord, lib.ko_job_coord_formula):
            fn.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p]
        lib.ko_rank.argtypes = [_f64p, ctypes.c_int64, _i64p, _i64p, _i64p]
        lib.ko_rank.restype = ctypes.c_int
        lib.ko_allpairs.argtypes = [
            _f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
            ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _i64p, _i64p, _i64p, _i64p, _i64p,
            _f64p,
        ]
        lib.ko_allpairs.restype = ctypes.c_int
        lib.ko_rect.argtypes = [
            _f64p, ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64, ctypes.c_int64,
            ctypes.c_int64, _i64p, _i64p, _i64p, _i64p, _f64p,
        ]
        lib.ko_rect.restype = ctypes.c_int
        _lib = lib
    return _lib


def _as_f64(x) -> np.ndarray:
    a = np.asarray(x)
    if a.dtype.kind == "f" and np.isnan(a).any():
        raise ValueError("NaN in oracle input")
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


def pair_counts(u, v, method: str = "definition") -> dict:
    """Counts for one pair: nc, nd, n1 (ties in u), n2 (ties in v), n3 (joint ties), S."""
    lib = _load()
    uu, vv = _as_f64(u), _as_f64(v)
    if uu.shape != vv.shape or uu.ndim != 1:
        raise ValueError("u and v must be 1-D of equal length")
    c = _Counts()
    if method == "definition":
        lib.ko_pair_definition(_ptr(uu, _f64p), _ptr(vv, _f64p), uu.size, ctypes.byref(c))
    elif method == "knight":
        if lib.ko_pair_knight(_ptr(uu, _f64p), _ptr(vv, _f64p), uu.size, ctypes.byref(c)) != 0:
            raise MemoryError
    else:
        raise ValueError(method)
    d = {k: int(getattr(c, k)) for k in ("nc", "nd", "n1", "n2", "n3")}
    d["S"] = d["nc"] - d["nd"]
    return d


def tau_b(S: int, n1: int, n2: int, n: int) -> float:
    """Eq. 3 in FP64; NaN when a variable is constant."""
    return float(_load().ko_tau_b(int(S), int(n1), int(n2), int(n)))


def tau_a(S: int, n: int) -> float:
    """Kendall's tau-a (Sec. 2: (n_c - n_d) / n_0, no tie correction) in FP64: the IEEE quotient
    of the two integers (Python's int / int is correctly rounded)."""
    n0 = n * (n - 1) // 2
    return int(S) / n0


def rn32(num: int, den: int) -> np.float32:
    """num / den rounded to the nearest FP32 value, ties to even, computed exactly with integers
    (normal range only)."""
    num, den = int(num), int(den)
    if den <= 0:
        raise ValueError("den must be positive")
    if num == 0:
        return np.float32(0.0)
    sign = -1 if num < 0 else 1
    x = Fraction(abs(num), den)
    e = abs(num).bit_length() - den.bit_length()  # 2^(e-1) < x < 2^(e+1)
    while x < Fraction(2) ** e:
        e -= 1
    while x >= Fraction(2) ** (e + 1):
        e += 1
    if not -126 <= e <= 127:
        raise ValueError("outside the normal FP32 range")
    mant = x / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q = mant.numerator // mant.denominator
    r = mant - q
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q % 2 == 1):
        q += 1
    if q == 1 << 24:
        q, e = 1 << 23, e + 1
    return np.float32(sign * float(Fraction(q) * Fraction(2) ** (e - 23)))


def tau_a32(S: int, n: int) -> np.float32:
    """FP32 tau-a: S / n_0 correctly rounded to FP32."""
    return rn32(int(S), n * (n - 1) // 2)


def job_id(m: int, y: int, x: int) -> int:
    return int(_load().ko_job_id(m, y, x))


def _coord(fn, m, J):
    y, x = ctypes.c_int64(), ctypes.c_int64()
    fn(m, J, ctypes.byref(y), ctypes.byref(x))
    return int(y.value), int(x.value)


def job_coord(m: int, J: int):
    """Eq. 9-10 plus integer check of Eq. 6 (diagonal-included numbering)."""
    return _coord(_load().ko_job_coord, m, J)


def job_coord_formula(m: int, J: int):
    """Eq. 9-10 exactly as printed, evaluated in FP64."""
    return _coord(_load().ko_job_coord_formula, m, J)


def rank(x):
    """Rank transform of one variable: (perm, rank, T)."""
    xx = _as_f64(x)
    n = xx.size
    perm = np.empty(n, np.int64)
    rk = np.empty(n, np.int64)
    T = ctypes.c_int64()
    if _load().ko_rank(_ptr(xx, _f64p), n, _ptr(perm, _i64p), _ptr(rk, _i64p), ctypes.byref(T)):
        raise MemoryError
    return perm, rk, int(T.value)


def allpairs(X, method: str = "knight", q: int = 8, threads: int = 1, p_begin: int = 0,
             p_end: int | None = None) -> dict:
    """Every pair (i<j) of the rows of X with packed index in [p_begin, p_end)."""
    XX = _as_f64(X)
    m, n = XX.shape
    P = m * (m - 1) // 2
    if p_end is None:
        p_end = P
    cnt = max(0, p_end - p_begin)
    out = {k: np.zeros(cnt, np.int64) for k in ("S", "n3", "nd", "n1", "n2")}
    out["tau"] = np.zeros(cnt, np.float64)
    rc = _load().ko_allpairs(
        _ptr(XX, _f64p), m, n, n, 0 if method == "definition" else 1, q, threads, p_begin, p_end,
        *(_ptr(out[k], _i64p) for k in ("S", "n3", "nd", "n1", "n2")), _ptr(out["tau"], _f64p),
    )
    if rc:
        raise MemoryError
    return out


def permutation_exceed(X, perms, p_begin: int = 0, p_end: int | None = None) -> np.ndarray:
    """Permutation test of independence for every pair i < j (Sec. 2: tau measures association;
    its significance under random relabelling of one variable). For each permutation sigma (a row
    of `perms`) the samples of the second variable are reordered, x_j -> x_j[sigma], and the pair
    counts one exceedance when |S(x_i, x_j[sigma])| >= |S(x_i, x_j)|. Counting is Knight's method
    through rect(); returns the exceedance counts of the packed pairs in [p_begin, p_end)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    P = m * (m - 1) // 2
    if p_end is None:
        p_end = P
    S_obs = allpairs(X, method="knight", p_begin=p_begin, p_end=p_end)["S"]
    iu, ju = np.triu_indices(m, 1)  # packed order: row-major strict upper triangle
    iu, ju = iu[p_begin:p_end], ju[p_begin:p_end]
    exceed = np.zeros(p_end - p_begin, np.int64)
    for sigma in np.asarray(perms):
        S_perm = rect(X, X[:, sigma.astype(np.int64)])["S"]  # [i][j]: x_i vs x_j[sigma]
        exceed += np.abs(S_perm[iu, ju]) >= np.abs(S_obs)
    return exceed


def rect(Q, D) -> dict:
    """Every row of Q against every row of D (Knight counting); arrays of shape [b, mdb]."""
    QQ, DD = _as_f64(Q), _as_f64(D)
    b, n = QQ.shape
    mdb, n2 = DD.shape
    if n != n2:
        raise ValueError("sample counts differ")
    out = {k: np.zeros((b, mdb), np.int64) for k in ("S", "n3", "n1", "n2")}
    out["tau"] = np.zeros((b, mdb), np.float64)
    rc = _load().ko_rect(
        _ptr(QQ, _f64p), b, n, _ptr(DD, _f64p), mdb, n, n,
        *(_ptr(out[k], _i64p) for k in ("S", "n3", "n1", "n2")), _ptr(out["tau"], _f64p),
    )
    if rc:
        raise MemoryError
    return out


def topk_order(S_row, Du: int, Dv_row, k: int):
    """Exact order of one query's database rows by |tau| = |S| / sqrt(Du * Dv), descending.

    Rows whose tau is NaN (Du == 0 or Dv == 0) come last; equal |tau| (as exact rationals
    S^2 / (Du * Dv)) keep the smaller row index first. Returns the first k row indices."""
    keyed = []
    for j, (s, dv) in enumerate(zip(S_row, Dv_row)):
        s, dv = int(s), int(dv)
        if Du == 0 or dv == 0:
            keyed.append((1, Fraction(0), j))
        else:
            keyed.append((0, -Fraction(s * s, dv), j))
    keyed.sort()
    return [j for _, _, j in keyed[:k]]


def query_topk(Q, D, k: int):
    """Oracle of the query form: full rect() results plus exact top-k per query row."""
    r = rect(Q, D)
    n = np.asarray(Q).shape[1]
    n0 = n * (n - 1) // 2
    b = r["S"].shape[0]
    idx = np.zeros((b, k), np.int64)
    tau = np.zeros((b, k), np.float64)
    for i in range(b):
        Du = n0 - int(r["n1"][i, 0]) if r["n1"].shape[1] else n0
        Dv = n0 - r["n2"][i]
        order = topk_order(r["S"][i], Du, Dv, k)
        idx[i, : len(order)] = order
        tau[i, : len(order)] = r["tau"][i, order]
    r["topk_idx"] = idx
    r["topk_tau"] = tau
    return r
