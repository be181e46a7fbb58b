"""Argument checks of the C ABI, run without a device.

Every entry point validates its sizes, pointers and shares on the host
before it touches the GPU, and returns a status (tc_count: TC_COUNT_ERROR)
with tc_last_error() set.  The calls below all stop in those checks, or
finish with nothing to count, so no CUDA call is made."""
import ctypes
import os
import shutil

import pytest

I32, I64, P = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
OK, INVALID, ID_RANGE, OVERFLOW = 0, 1, 2, 6
TOP = (1 << 31) - (1 << 10)  # largest m and n a run accepts
ERR = (1 << 64) - 1          # TC_COUNT_ERROR


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1503_00576_gb300 import build

    so = ctypes.CDLL(build.build())
    sig = {
        "tc_count": (ctypes.c_uint64, [P, P, I64, I32, P]),
        "tc_count_per_vertex": (I32, [P, P, I64, I32, P, P, P, P]),
        "tc_count_part": (I32, [P, P, I64, I32, I32, I32, P, P]),
        "tc_count_host": (I32, [P, P, I64, I32, P]),
        "tc_count_per_vertex_host": (I32, [P, P, I64, I32, P, P, P]),
        "tc_count_ws": (I32, [P, P, I64, I32, P, P, ctypes.c_size_t, P]),
        "tc_count_noalloc": (I32, [P, P, I64, I32, P, P]),
        "tc_count_batch": (I32, [P, P, I32, P, P, P, P]),
        "tc_count_work_part": (I32, [P, P, I64, I32, I32, I32, P, P]),
        "tc_engine_create": (I32, [I64, I32, I32, P, P]),
        "tc_last_error": (I32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(so, name)
        f.restype, f.argtypes = res, args
    return so


def status(lib, rc):
    assert rc == lib.tc_last_error()
    return rc


def arr(ctype, values):
    return (ctype * len(values))(*values)


def test_single_graph_sizes(lib):
    pairs = arr(I32, [0, 1, 2])
    assert lib.tc_count(None, None, -1, 5, None) == ERR and lib.tc_last_error() == INVALID
    assert lib.tc_count(None, None, 5, -1, None) == ERR and lib.tc_last_error() == INVALID
    assert lib.tc_count(None, None, TOP + 1, 5, None) == ERR and lib.tc_last_error() == OVERFLOW
    assert lib.tc_count(None, None, 5, TOP + 1, None) == ERR and lib.tc_last_error() == OVERFLOW
    # the padded lists of m = n = 2^31 - 2^10 would need 2^34 words
    assert lib.tc_count(None, None, TOP, TOP, None) == ERR and lib.tc_last_error() == OVERFLOW
    assert lib.tc_count(None, None, 3, 5, None) == ERR and lib.tc_last_error() == INVALID
    # pairs but no vertex: every id is out of range
    assert lib.tc_count(pairs, pairs, 3, 0, None) == ERR and lib.tc_last_error() == ID_RANGE


def test_outputs_and_shares(lib):
    total = ctypes.c_uint64(7)
    assert status(lib, lib.tc_count_per_vertex(None, None, 0, 4, None, None, None, None)) == INVALID
    assert status(lib, lib.tc_count_part(None, None, 0, 4, 0, 2, None, None)) == INVALID
    for part, parts in [(2, 2), (-1, 2), (0, 0)]:
        rc = lib.tc_count_part(None, None, 0, 4, part, parts, None, ctypes.byref(total))
        assert status(lib, rc) == INVALID
    assert status(lib, lib.tc_count_host(None, None, 3, 4, ctypes.byref(total))) == INVALID
    rc = lib.tc_count_per_vertex_host(None, None, 0, 4, None, None, ctypes.byref(total))
    assert status(lib, rc) == INVALID
    rc = lib.tc_count_ws(None, None, 0, 4, None, None, 0, ctypes.byref(total))
    assert status(lib, rc) == INVALID
    assert status(lib, lib.tc_count_work_part(None, None, 0, 4, 0, 1, None, None)) == INVALID


def test_allocation_free_entry(lib):
    total = ctypes.c_uint64(7)
    pairs = arr(I32, [0])
    assert status(lib, lib.tc_count_noalloc(None, None, 0, 4, None, None)) == INVALID
    assert status(lib, lib.tc_count_noalloc(None, None, 0, 4, None, ctypes.byref(total))) == OK
    assert total.value == 0
    # ten million pairs need far more than the static scratch holds
    rc = lib.tc_count_noalloc(pairs, pairs, 10 ** 7, 10 ** 6, None, ctypes.byref(total))
    assert status(lib, rc) == OVERFLOW


def test_batches(lib):
    totals = arr(ctypes.c_uint64, [9, 9, 9])
    assert status(lib, lib.tc_count_batch(None, None, -1, None, None, None, totals)) == INVALID
    assert status(lib, lib.tc_count_batch(None, None, 2, None, None, None, totals)) == INVALID
    bad = [([1, 2, 3], [4, 4]), ([0, 3, 2], [4, 4]), ([0, 1, 2], [4, -4])]
    for eo, vn in bad:
        rc = lib.tc_count_batch(None, None, 2, arr(I64, eo), arr(I32, vn), None, totals)
        assert status(lib, rc) == INVALID
    big = [([0, TOP + 1], [4]), ([0, 1, 2], [TOP, 1 << 10])]
    for eo, vn in big:
        g = len(vn)
        rc = lib.tc_count_batch(None, None, g, arr(I64, eo), arr(I32, vn), None, totals)
        assert status(lib, rc) == OVERFLOW
    rc = lib.tc_count_batch(None, None, 2, arr(I64, [0, 1, 2]), arr(I32, [4, 4]), None, None)
    assert status(lib, rc) == INVALID
    # graphs without pairs: every total is 0, nothing to run
    rc = lib.tc_count_batch(None, None, 3, arr(I64, [0, 0, 0, 0]), arr(I32, [0, 5, 9]), None, totals)
    assert status(lib, rc) == OK and list(totals) == [0, 0, 0]
    assert status(lib, lib.tc_count_batch(None, None, 0, None, None, None, None)) == OK


def test_engine_capacities(lib):
    out = ctypes.c_void_p(1)
    assert status(lib, lib.tc_engine_create(1, 1, 1, None, None)) == INVALID
    for caps in [(0, 1, 1), (1, 0, 1), (1, 1, 0), (-5, 1, 1)]:
        assert status(lib, lib.tc_engine_create(*caps, None, ctypes.byref(out))) == INVALID
        assert out.value is None
    for caps in [(TOP + 1, 1, 1), (1, TOP + 1, 1), (TOP, TOP, 1)]:
        assert status(lib, lib.tc_engine_create(*caps, None, ctypes.byref(out))) == OVERFLOW
        assert out.value is None
