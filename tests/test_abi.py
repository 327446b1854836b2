"""Host-side checks of the C ABI: the library loads, exports every function that
include/ktau.h declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ktau.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03767_gb300 import build as kb

    kb.build()
    import paper_1704_03767_gb300 as ktau

    return ktau.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ktau_[a-z_0-9]+)\s*\(", src)))


def test_header_parses():
    names = _declared()
    for must in ("ktau_rank_prepare", "ktau_allpairs", "ktau_query", "ktau_batch_create"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    import paper_1704_03767_gb300 as ktau

    names = _declared()
    bound = set(ktau.declared_symbols())
    for name in names:
        assert hasattr(lib, name), f"{name} not exported by libktau.so"
        assert name in bound, f"{name} has no binding"


def test_abi_version_and_status_strings(lib):
    assert lib.ktau_abi_version() == 1
    assert lib.ktau_status_string(0) == b"KTAU_OK"
    assert lib.ktau_status_string(2) == b"KTAU_ENAN"


def test_argument_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    # NULL values
    assert lib.ktau_rank_prepare(None, 0, 10, 10, 10, None, ctypes.byref(h)) == 1
    # bad dtype
    assert lib.ktau_rank_prepare(fake, 7, 10, 10, 10, None, ctypes.byref(h)) == 1
    # m < 1, n < 2, ld < n
    assert lib.ktau_rank_prepare(fake, 0, 0, 10, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare(fake, 0, 10, 1, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare(fake, 0, 10, 10, 9, None, ctypes.byref(h)) == 1
    # n beyond the 16-bit rank storage
    assert lib.ktau_rank_prepare(fake, 0, 10, 16385, 16385, None, ctypes.byref(h)) == 3
    assert b"KTAU_MAX_N" in lib.ktau_last_error()
    assert h.value is None
    # the asynchronous form validates the same way before any device work
    assert lib.ktau_rank_prepare_async(None, 0, 10, 10, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 7, 10, 10, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 0, 10, 10, 9, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 0, 10, 16385, 16385, None, ctypes.byref(h)) == 3
    assert h.value is None
    # trace filter: host state only
    assert lib.ktau_trace_filter(b"contract_kernel") == 0
    assert lib.ktau_trace_filter(None) == 0
    # NULL handle
    assert lib.ktau_allpairs(None, 0, 1, None, None, None, None, 32, None, None) == 1
    assert lib.ktau_query(None, None, None, None, None, 32, 0, None, None, None, None) == 1
    assert lib.ktau_ranked_free(None) == 0
