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
    assert lib.ktau_abi_version() == 2
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
    # n beyond KTAU_MAX_N = 4194304 (rows above 65535 samples keep 32-bit ranks)
    big = 4194305
    assert lib.ktau_rank_prepare(fake, 0, 10, big, big, None, ctypes.byref(h)) == 3
    assert b"KTAU_MAX_N" in lib.ktau_last_error()
    assert h.value is None
    # the asynchronous form validates the same way before any device work
    assert lib.ktau_rank_prepare_async(None, 0, 10, 10, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 7, 10, 10, 10, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 0, 10, 10, 9, None, ctypes.byref(h)) == 1
    assert lib.ktau_rank_prepare_async(fake, 0, 10, big, big, None, ctypes.byref(h)) == 3
    assert h.value is None
    # trace filter: host state only
    assert lib.ktau_trace_filter(b"contract_kernel") == 0
    assert lib.ktau_trace_filter(None) == 0
    # NULL handle
    assert lib.ktau_allpairs(None, 0, 1, None, None, None, None, 32, None, None) == 1
    assert lib.ktau_query(None, None, None, None, None, 32, 0, None, None, None, None) == 1
    assert lib.ktau_ranked_free(None) == 0


def test_workspace_size_without_gpu(lib):
    """ktau_workspace_size is host arithmetic only: it runs without a GPU, grows with the
    datasets, and covers at least the three rank arrays of every dataset."""
    import paper_1704_03767_gb300 as ktau

    def desc(m, n, path=1):
        return ktau.BatchDesc(0x1000, 0, 32, m, n, n, None, None, None, None, path, 0)

    small = ktau.ktau_workspace_size([desc(10, 20)])
    big = ktau.ktau_workspace_size([desc(10, 20), desc(300, 500)])
    assert small >= 3 * 10 * 32 * 2 and big > small
    # contraction datasets also hold their sign operands: packed FP4 by default, n_0 rounded up to
    # 256 elements (128 bytes) per row; FP8 takes twice that
    sg = ktau.ktau_workspace_size([desc(300, 100, 2)])
    assert sg >= 300 * ((100 * 99 // 2 + 255) // 256 * 128)
    opt8 = ktau.Options()
    opt8.operand_bits = 8
    sg8 = ktau.ktau_workspace_size([desc(300, 100, 2)], options=opt8)
    assert sg8 >= 300 * ((100 * 99 // 2 + 127) // 128 * 128) and sg8 > sg
    size = ctypes.c_size_t()
    assert lib.ktau_workspace_size(None, 1, None, ctypes.byref(size)) == 1
    arr = (ktau.BatchDesc * 1)(desc(1, 20))  # m < 2
    assert lib.ktau_workspace_size(arr, 1, None, ctypes.byref(size)) == 1
    arr = (ktau.BatchDesc * 1)(desc(10, 20))
    assert lib.ktau_workspace_size(arr, 1, None, None) == 1
    # the batched call rejects a missing or unaligned workspace before any device work
    assert lib.ktau_allpairs_batched(arr, 1, None, None, 1 << 20, None, None) == 1
    assert lib.ktau_allpairs_batched(arr, 1, None, 0x1001, 1 << 20, None, None) == 1
    # p-values: B < 0 and NULL arrays
    assert lib.ktau_permutation_pvalues(None, -1, 5, None, None) == 1
    assert lib.ktau_permutation_pvalues(None, 3, 5, None, None) == 1
    assert lib.ktau_permutation_pvalues(None, 3, 0, None, None) == 0
