"""ctypes binding of libktau.so (include/ktau.h). Argument marshalling only: every step of the
computation runs in the library's CUDA kernels. Torch provides device memory and streams.

Functions keep the C names. Handles are wrapped so that they are freed with their owner.
If the library has not been built, importing raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libktau.so")

KTAU_OK, KTAU_EINVAL, KTAU_ENAN, KTAU_ETOOLARGE, KTAU_ENOMEM, KTAU_ECUDA, KTAU_ETIMEOUT, \
    KTAU_EBUSY = range(8)
KTAU_F32, KTAU_I32 = 0, 1
KTAU_PATH_AUTO, KTAU_PATH_MERGE, KTAU_PATH_SIGNGEMM, KTAU_PATH_BITS = 0, 1, 2, 3
KTAU_BITS_MAX_N = 256
KTAU_MAX_N = 4194304
KTAU_NARROW_MAX_N = 65535
KTAU_BATCH_MAX_N = 16384

STATUS_NAMES = {0: "KTAU_OK", 1: "KTAU_EINVAL", 2: "KTAU_ENAN", 3: "KTAU_ETOOLARGE",
                4: "KTAU_ENOMEM", 5: "KTAU_ECUDA", 6: "KTAU_ETIMEOUT", 7: "KTAU_EBUSY"}


class KtauError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_q", ctypes.c_int32),
                ("mapping", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("operand_bits", ctypes.c_int32),
                ("statistic", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class TraceRecord(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("ms", ctypes.c_float)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("dtype", ctypes.c_int32),
                ("count_bits", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("tau64", ctypes.c_void_p), ("tau32", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("n3", ctypes.c_void_p), ("path", ctypes.c_int32),
                ("mapping", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32, _i64, _u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_SIGS = {
    "ktau_last_error": ([], ctypes.c_char_p),
    "ktau_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "ktau_abi_version": ([], _i32),
    "ktau_rank_prepare": ([_vp, ctypes.c_int, _i64, _i64, _i64, _vp, ctypes.POINTER(_vp)],
                          ctypes.c_int),
    "ktau_rank_prepare_async": ([_vp, ctypes.c_int, _i64, _i64, _i64, _vp, ctypes.POINTER(_vp)],
                                ctypes.c_int),
    "ktau_rank_prepare_host": ([_vp, ctypes.c_int, _i64, _i64, _i64, _vp, ctypes.POINTER(_vp)],
                               ctypes.c_int),
    "ktau_ranked_free": ([_vp], ctypes.c_int),
    "ktau_ranked_free_on": ([_vp, _vp], ctypes.c_int),
    "ktau_ranked_shape": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
    "ktau_tie_counts": ([_vp, _vp, _vp], ctypes.c_int),
    "ktau_ranked_export": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "ktau_ranked_export32": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "ktau_allpairs": ([_vp, _u64, _u64, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(Options), _vp],
                      ctypes.c_int),
    "ktau_allpairs_noalloc": ([_vp, ctypes.c_int, _i64, _i64, _i64, _u64, _u64, _vp, _vp, _vp,
                               _vp, _i32, _vp], ctypes.c_int),
    "ktau_allpairs_host": ([_vp, _u64, _u64, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(Options),
                            _u64, _vp], ctypes.c_int),
    "ktau_allpairs_path": ([_vp, ctypes.POINTER(Options), ctypes.POINTER(_i32)], ctypes.c_int),
    "ktau_prepare_signs": ([_vp, _vp], ctypes.c_int),
    "ktau_device_status": ([_vp], ctypes.c_int),
    "ktau_permutation_exceed": ([_vp, _vp, _i32, _u64, _u64, _vp, _vp, _vp], ctypes.c_int),
    "ktau_permutation_pvalues": ([_vp, _i32, _u64, _vp, _vp], ctypes.c_int),
    "ktau_debug_fail_alloc": ([_i32], ctypes.c_int),
    "ktau_debug_wait_timeout": ([_i64, _vp], ctypes.c_int),
    "ktau_trace_enable": ([_i32], ctypes.c_int),
    "ktau_trace_filter": ([ctypes.c_char_p], ctypes.c_int),
    "ktau_trace_collect": ([ctypes.POINTER(TraceRecord), _i32, ctypes.POINTER(_i32)],
                           ctypes.c_int),
    "ktau_batch_create": ([ctypes.POINTER(BatchDesc), _i32, ctypes.POINTER(Options),
                           ctypes.POINTER(_vp)], ctypes.c_int),
    "ktau_batch_run": ([_vp, _vp], ctypes.c_int),
    "ktau_batch_graph_launch": ([_vp, _vp], ctypes.c_int),
    "ktau_batch_check": ([_vp, _vp], ctypes.c_int),
    "ktau_batch_paths": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], ctypes.c_int),
    "ktau_batch_pairs": ([_vp, ctypes.POINTER(_u64)], ctypes.c_int),
    "ktau_batch_free": ([_vp], ctypes.c_int),
    "ktau_allpairs_batched": ([ctypes.POINTER(BatchDesc), _i32, ctypes.POINTER(Options), _vp,
                               ctypes.c_size_t, _vp, _vp], ctypes.c_int),
    "ktau_workspace_size": ([ctypes.POINTER(BatchDesc), _i32, ctypes.POINTER(Options),
                             ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "ktau_query": ([_vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp, ctypes.POINTER(Options), _vp],
                   ctypes.c_int),
    "ktau_query_scratch_bytes": ([_vp, _i64, _i32, ctypes.POINTER(ctypes.c_size_t)],
                                 ctypes.c_int),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libktau.so (raises if it is missing: build it with paper_1704_03767_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing; run `python -m paper_1704_03767_gb300.build`")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(status: int):
    if status != KTAU_OK:
        raise KtauError(status, load().ktau_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _options(options):
    if options is None:
        return None
    if isinstance(options, Options):
        return ctypes.byref(options)
    o = Options()
    for k, v in dict(options).items():
        setattr(o, k, int(v))
    return ctypes.byref(o)


class Ranked:
    """Owner of a ktau_ranked handle (device-resident ranks of an m x n matrix)."""

    def __init__(self, handle: int, m: int, n: int, device: torch.device):
        self.handle = handle
        self.m, self.n = m, n
        self.device = device

    @property
    def pairs(self) -> int:
        return self.m * (self.m - 1) // 2

    def free(self):
        if self.handle:
            load().ktau_ranked_free(self.handle)
            self.handle = None

    def free_on(self, stream):
        """Release after synchronising only `stream` (all uses of the handle were on it)."""
        if self.handle:
            _check(load().ktau_ranked_free_on(self.handle, _stream(stream)))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ktau_rank_prepare(values: torch.Tensor, stream=None) -> Ranked:
    """Rank transform of every row of a CUDA float32/int32 matrix (row-major, unit column stride)."""
    return _rank_prepare(values, stream, "ktau_rank_prepare")


def ktau_rank_prepare_async(values: torch.Tensor, stream=None) -> Ranked:
    """ktau_rank_prepare without synchronising the stream: a NaN is reported (KtauError, status 2)
    by the first call that uses the handle. `values` must stay alive until the stream has run
    the rank transform."""
    return _rank_prepare(values, stream, "ktau_rank_prepare_async")


def ktau_rank_prepare_host(values: torch.Tensor, stream=None, device=None) -> Ranked:
    """Rank transform of a HOST float32/int32 matrix (pinned for full copy bandwidth): the library
    copies it to the device and ranks it there."""
    if values.dim() != 2 or values.is_cuda:
        raise ValueError("values must be a 2-D host tensor")
    return _rank_prepare(values, stream, "ktau_rank_prepare_host",
                         device or torch.device("cuda", torch.cuda.current_device()))


def _rank_prepare(values: torch.Tensor, stream, fn: str, device=None) -> Ranked:
    if values.dim() != 2 or (device is None and not values.is_cuda):
        raise ValueError("values must be a 2-D CUDA tensor")
    if values.dtype == torch.float32:
        dt = KTAU_F32
    elif values.dtype == torch.int32:
        dt = KTAU_I32
    else:
        raise ValueError("values must be float32 or int32")
    if values.stride(1) != 1:
        raise ValueError("values must have unit column stride")
    m, n = values.shape
    h = ctypes.c_void_p()
    _check(getattr(load(), fn)(values.data_ptr(), dt, m, n, values.stride(0), _stream(stream),
                               ctypes.byref(h)))
    return Ranked(h.value, m, n, device or values.device)


def ktau_tie_counts(R: Ranked, T: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if T is None:
        T = torch.empty(R.m, dtype=torch.int64, device=R.device)
    _check(load().ktau_tie_counts(R.handle, T.data_ptr(), _stream(stream)))
    return T


def ktau_ranked_export(R: Ranked, stream=None):
    perm = torch.empty((R.m, R.n), dtype=torch.uint16, device=R.device)
    rank = torch.empty((R.m, R.n), dtype=torch.uint16, device=R.device)
    _check(load().ktau_ranked_export(R.handle, perm.data_ptr(), rank.data_ptr(), _stream(stream)))
    return perm, rank


def ktau_ranked_export32(R: Ranked, stream=None):
    """perm and rank as 32-bit rows (any n). Returned as int32 tensors holding the uint32 values,
    which are below 2^31 for every n the library takes."""
    perm = torch.empty((R.m, R.n), dtype=torch.int32, device=R.device)
    rank = torch.empty((R.m, R.n), dtype=torch.int32, device=R.device)
    _check(load().ktau_ranked_export32(R.handle, perm.data_ptr(), rank.data_ptr(),
                                       _stream(stream)))
    return perm, rank


def ktau_allpairs(R: Ranked, p_begin: int = 0, p_end: int | None = None, tau64=None, tau32=None,
                  S=None, n3=None, count_bits: int = 32, options=None, stream=None):
    """Enqueues tau-b for pairs [p_begin, p_end) into the given CUDA tensors (any may be None)."""
    if p_end is None:
        p_end = R.pairs
    _check(load().ktau_allpairs(R.handle, p_begin, p_end, _ptr(tau64), _ptr(tau32), _ptr(S),
                                _ptr(n3), count_bits, _options(options), _stream(stream)))


def ktau_allpairs_noalloc(values: torch.Tensor, p_begin: int = 0, p_end: int | None = None,
                          tau64=None, tau32=None, S=None, n3=None, count_bits: int = 32,
                          stream=None):
    """ktau_allpairs for one matrix from its values, using only the library's fixed scratch."""
    if values.dim() != 2 or not values.is_cuda or values.stride(1) != 1:
        raise ValueError("values must be a 2-D CUDA tensor with unit column stride")
    dt = KTAU_F32 if values.dtype == torch.float32 else KTAU_I32
    m, n = values.shape
    if p_end is None:
        p_end = m * (m - 1) // 2
    _check(load().ktau_allpairs_noalloc(values.data_ptr(), dt, m, n, values.stride(0), p_begin,
                                        p_end, _ptr(tau64), _ptr(tau32), _ptr(S), _ptr(n3),
                                        count_bits, _stream(stream)))


def ktau_allpairs_host(R: Ranked, p_begin: int = 0, p_end: int | None = None, tau64=None,
                       tau32=None, S=None, n3=None, count_bits: int = 32, options=None,
                       pass_pairs: int = 0, stream=None):
    """ktau_allpairs into HOST tensors (pinned for full bandwidth), in passes whose copies overlap
    the next pass's compute. Returns when the host tensors are complete."""
    if p_end is None:
        p_end = R.pairs
    for t in (tau64, tau32, S, n3):
        if t is not None and t.is_cuda:
            raise ValueError("ktau_allpairs_host takes host tensors")
    _check(load().ktau_allpairs_host(R.handle, p_begin, p_end, _ptr(tau64), _ptr(tau32), _ptr(S),
                                     _ptr(n3), count_bits, _options(options), pass_pairs,
                                     _stream(stream)))


def ktau_allpairs_path(R: Ranked, options=None) -> int:
    p = ctypes.c_int32()
    _check(load().ktau_allpairs_path(R.handle, _options(options), ctypes.byref(p)))
    return p.value


def ktau_prepare_signs(R: Ranked, stream=None):
    _check(load().ktau_prepare_signs(R.handle, _stream(stream)))


def ktau_device_status(stream=None):
    _check(load().ktau_device_status(_stream(stream)))


def ktau_permutation_exceed(R: Ranked, perms: torch.Tensor, S_obs: torch.Tensor,
                            exceed: torch.Tensor, p_begin: int = 0, p_end: int | None = None,
                            stream=None):
    """Adds, per pair of [p_begin, p_end), the number of permutations (rows of `perms`, uint16
    [B, n] on the device) under which |S| of the relabelled pair reaches the observed |S|."""
    if p_end is None:
        p_end = R.pairs
    if perms.dtype != torch.uint16 or perms.dim() != 2 or perms.shape[1] != R.n:
        raise ValueError("perms must be a uint16 [B, n] tensor")
    if S_obs.dtype != torch.int32 or exceed.dtype != torch.uint32:
        raise ValueError("S_obs must be int32 and exceed uint32")
    _check(load().ktau_permutation_exceed(R.handle, perms.data_ptr(), perms.shape[0], p_begin,
                                          p_end, S_obs.data_ptr(), exceed.data_ptr(),
                                          _stream(stream)))


def permutation_pvalues(values: torch.Tensor, perms: torch.Tensor, stream=None):
    """Two-sided permutation p-values (exceed + 1) / (B + 1) of every pair (FP64, packed triangle),
    with the observed tau-b and S."""
    res = allpairs(values, want=("tau64", "S"), stream=stream)
    R = res["ranked"]
    exceed = torch.zeros(R.pairs, dtype=torch.uint32, device=values.device)
    ktau_permutation_exceed(R, perms.to(values.device), res["S"], exceed, stream=stream)
    res["exceed"] = exceed
    res["pvalue"] = ktau_permutation_pvalues(exceed, perms.shape[0], stream=stream)
    return res


def ktau_permutation_pvalues(exceed: torch.Tensor, B: int, pvalue=None, stream=None):
    """(exceed + 1) / (B + 1) per pair, computed by the library (FP64 CUDA tensor)."""
    if exceed.dtype != torch.uint32 or not exceed.is_cuda:
        raise ValueError("exceed must be a uint32 CUDA tensor")
    if pvalue is None:
        pvalue = torch.empty(exceed.numel(), dtype=torch.float64, device=exceed.device)
    _check(load().ktau_permutation_pvalues(exceed.data_ptr(), B, exceed.numel(),
                                           pvalue.data_ptr(), _stream(stream)))
    return pvalue


def ktau_debug_fail_alloc(k: int):
    _check(load().ktau_debug_fail_alloc(k))


def ktau_debug_wait_timeout(limit_ns: int, stream=None):
    _check(load().ktau_debug_wait_timeout(limit_ns, _stream(stream)))


def ktau_trace_enable(on: bool = True):
    _check(load().ktau_trace_enable(1 if on else 0))


def ktau_trace_filter(name: str | None = None):
    """Trace only the launches named `name` (None: every launch)."""
    _check(load().ktau_trace_filter(name.encode() if name else None))


def ktau_trace_collect(cap: int = 65536):
    """List of (kernel name, milliseconds) for the launches recorded since the last collect."""
    arr = (TraceRecord * cap)()
    n = ctypes.c_int32()
    _check(load().ktau_trace_collect(arr, cap, ctypes.byref(n)))
    return [(arr[i].name.decode(), float(arr[i].ms)) for i in range(n.value)]


def allpairs(values: torch.Tensor, p_begin: int = 0, p_end: int | None = None,
             count_bits: int = 32, want=("tau64", "tau32", "S", "n3"), options=None, stream=None):
    """Convenience: rank + all pairs with freshly allocated outputs (dict of tensors)."""
    R = ktau_rank_prepare(values, stream)
    if p_end is None:
        p_end = R.pairs
    cnt = p_end - p_begin
    dev = values.device
    cdt = torch.int32 if count_bits == 32 else torch.int64
    out = {}
    if "tau64" in want:
        out["tau64"] = torch.empty(cnt, dtype=torch.float64, device=dev)
    if "tau32" in want:
        out["tau32"] = torch.empty(cnt, dtype=torch.float32, device=dev)
    if "S" in want:
        out["S"] = torch.empty(cnt, dtype=cdt, device=dev)
    if "n3" in want:
        out["n3"] = torch.empty(cnt, dtype=cdt, device=dev)
    ktau_allpairs(R, p_begin, p_end, out.get("tau64"), out.get("tau32"), out.get("S"),
                  out.get("n3"), count_bits, options, stream)
    out["T"] = ktau_tie_counts(R, stream=stream)
    out["ranked"] = R
    return out


class Batch:
    """Owner of a ktau_batch plan (many matrices in one persistent launch per kernel family)."""

    def __init__(self, descs, options=None, keepalive=None):
        arr = (BatchDesc * len(descs))(*descs)
        h = ctypes.c_void_p()
        _check(load().ktau_batch_create(arr, len(descs), _options(options), ctypes.byref(h)))
        self.handle = h.value
        self._keepalive = keepalive

    def run(self, stream=None):
        _check(load().ktau_batch_run(self.handle, _stream(stream)))

    def graph_launch(self, stream=None):
        _check(load().ktau_batch_graph_launch(self.handle, _stream(stream)))

    def check(self, stream=None):
        _check(load().ktau_batch_check(self.handle, _stream(stream)))

    def paths(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(load().ktau_batch_paths(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def pairs(self) -> int:
        p = ctypes.c_uint64()
        _check(load().ktau_batch_pairs(self.handle, ctypes.byref(p)))
        return p.value

    def free(self):
        if self.handle:
            load().ktau_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_desc(values: torch.Tensor, tau64=None, tau32=None, S=None, n3=None,
               count_bits: int = 32, path: int = KTAU_PATH_AUTO, mapping: int = 0) -> BatchDesc:
    m, n = values.shape
    dt = KTAU_F32 if values.dtype == torch.float32 else KTAU_I32
    return BatchDesc(values.data_ptr(), dt, count_bits, m, n, values.stride(0), _ptr(tau64),
                     _ptr(tau32), _ptr(S), _ptr(n3), path, mapping)


def ktau_workspace_size(descs, options=None) -> int:
    """Bytes of device workspace ktau_allpairs_batched needs for these descriptors."""
    arr = (BatchDesc * len(descs))(*descs)
    v = ctypes.c_size_t()
    _check(load().ktau_workspace_size(arr, len(descs), _options(options), ctypes.byref(v)))
    return v.value


def ktau_allpairs_batched(descs, workspace: torch.Tensor, nan_flag=None, options=None,
                          stream=None):
    """Every dataset of `descs` in one call, with all scratch in `workspace` (a CUDA uint8 tensor
    of at least ktau_workspace_size bytes, 256-byte aligned); `nan_flag` is an optional CUDA
    int32/uint32 tensor of one element that receives the call's NaN flag."""
    arr = (BatchDesc * len(descs))(*descs)
    _check(load().ktau_allpairs_batched(arr, len(descs), _options(options), workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(),
                                        _ptr(nan_flag), _stream(stream)))


def ktau_query(db: Ranked, queries: Ranked, tau=None, S=None, n3=None, count_bits: int = 32,
               k: int = 0, topk_idx=None, topk_tau=None, options=None, stream=None):
    _check(load().ktau_query(db.handle, queries.handle, _ptr(tau), _ptr(S), _ptr(n3), count_bits,
                             k, _ptr(topk_idx), _ptr(topk_tau), _options(options),
                             _stream(stream)))


def ktau_query_scratch_bytes(db: Ranked, b: int, k: int) -> int:
    v = ctypes.c_size_t()
    _check(load().ktau_query_scratch_bytes(db.handle, b, k, ctypes.byref(v)))
    return v.value
