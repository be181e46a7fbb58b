"""The C-ABI library builds, loads and exports every symbol of include/*.h.

CPU only: nothing here calls into the GPU code (no device is needed to load
the shared library, and no compute entry point is invoked)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def header_functions():
    names = set()
    for path in HEADERS:
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^[A-Za-z_][\w \*]*?\b(tc_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1503_00576_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_lists_the_api():
    names = header_functions()
    assert [os.path.basename(h) for h in HEADERS] == ["tc.h", "tc_debug.h"]
    assert "tc_count" in names and "tc_count_per_vertex" in names
    assert "tc_debug_set_wait_limit" in names
    assert len(names) >= 12


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    import paper_1503_00576_gb300 as tc

    assert sorted(tc.EXPORTS) == header_functions()


def test_pure_host_entry_points(lib):
    """Entry points that touch no device: names and sizes."""
    lib.tc_status_string.restype = ctypes.c_char_p
    assert lib.tc_status_string(0) == b"ok"
    assert lib.tc_status_string(2) == b"vertex id out of range"
    lib.tc_phase_name.restype = ctypes.c_char_p
    assert [lib.tc_phase_name(i) for i in range(8)] == [
        b"canon", b"rank", b"orient", b"sort", b"offsets", b"lists", b"groups", b"count"]
    lib.tc_workspace_bytes.restype = ctypes.c_size_t
    lib.tc_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
    small = lib.tc_workspace_bytes(1000, 100)
    big = lib.tc_workspace_bytes(10 ** 8, 1 << 24)
    assert 0 < small < big
    assert big >= 2 * 8 * 10 ** 8  # two key buffers of 8 bytes per pair
    assert lib.tc_workspace_bytes(-1, 5) == 0
    assert lib.tc_workspace_bytes(1 << 31, 5) == 0
    # the limits: 2^31 - 2^10 pairs and vertices, one more is refused
    top = (1 << 31) - (1 << 10)
    assert lib.tc_workspace_bytes(top, 5) > 16 * top
    assert lib.tc_workspace_bytes(top + 1, 5) == 0
    assert lib.tc_workspace_bytes(5, top) > lib.tc_workspace_bytes(5, 1 << 20)
    assert lib.tc_workspace_bytes(5, top + 1) == 0


def test_missing_library_fails_loudly(tmp_path):
    import paper_1503_00576_gb300 as tc

    saved = tc._lib
    tc._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            tc.load_library(str(tmp_path / "missing.so"))
    finally:
        tc._lib = saved
