"""The allocation-free entry point against the ordinary one and the oracle.

tc_count_noalloc serves callers that cannot allocate device memory while
they run (their own allocator owns the device memory, or their memory budget
is fixed at start-up).  It must count exactly what tc_count counts -- the
counts are integers, so the tolerance is zero -- on two calls in a row, since
every call reuses the same static scratch array, and what the CPU oracle
counts.  A warm call must take no device memory: with every library
allocation made to fail, and with the device's free memory unchanged.  This
file sorts last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1503_00576_gb300 as lib

    lib.load_library()
    return lib


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def _noalloc(tc, s, d, n):
    """Direct C-ABI call: returns (status, T)."""
    import torch

    lib = tc.load_library()
    total = ctypes.c_uint64(0)
    rc = lib.tc_count_noalloc(s.data_ptr(), d.data_ptr(), s.numel(), n,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                              ctypes.byref(total))
    return rc, int(total.value)


@pytest.mark.parametrize("scale,seed", [(16, 5), (12, 6)])
def test_matches_tc_count_twice(tc, scale, seed):
    src, dst = graphgen.rmat(scale, 16 << scale, seed)
    n = 1 << scale
    s, d = _dev(src), _dev(dst)
    want = tc.tc_count(s, d, n)
    assert want > 0
    for _ in range(2):
        rc, got = _noalloc(tc, s, d, n)
        assert rc == tc.TC_OK, tc.load_library().tc_last_error_detail()
        assert got == want


def test_different_graphs_back_to_back(tc):
    """The scratch keeps the previous call's contents; results must not
    depend on them."""
    a = graphgen.rmat(15, 16 << 15, 9)
    b = graphgen.er(20000, 200000, 10)
    ga = (_dev(a[0]), _dev(a[1]), 1 << 15)
    gb = (_dev(b[0]), _dev(b[1]), 20000)
    want = [tc.tc_count(*ga), tc.tc_count(*gb)]
    got = [_noalloc(tc, *ga), _noalloc(tc, *gb), _noalloc(tc, *ga)]
    assert [g[0] for g in got] == [tc.TC_OK] * 3
    assert [g[1] for g in got] == [want[0], want[1], want[0]]


def test_rejects_oversize_then_recovers(tc):
    src, dst = graphgen.rmat(18, 16 << 18, 11)  # needs ~100 MB of scratch
    s, d = _dev(src), _dev(dst)
    rc, _ = _noalloc(tc, s, d, 1 << 18)
    assert rc == tc.TC_ERR_OVERFLOW
    assert b"static scratch holds" in tc.load_library().tc_last_error_detail()
    small = graphgen.rmat(10, 16 << 10, 12)
    assert tc.tc_count_noalloc(_dev(small[0]), _dev(small[1]), 1 << 10) == \
        tc.tc_count(_dev(small[0]), _dev(small[1]), 1 << 10)


def test_matches_the_oracle(tc):
    src, dst = graphgen.rmat(14, 16 << 14, 21)
    n = 1 << 14
    want = oracle.forward(src, dst, n, per_vertex=False)["T"]
    s, d = _dev(src), _dev(dst)
    for _ in range(2):
        rc, got = _noalloc(tc, s, d, n)
        assert rc == tc.TC_OK
        assert got == want


def test_warm_call_takes_no_device_memory(tc):
    """After a first (warm-up) call on the device, a call allocates nothing:
    it succeeds while every allocation the library could make is set to
    fail, and the device's free memory does not move."""
    import torch

    src, dst = graphgen.rmat(13, 16 << 13, 22)
    n = 1 << 13
    s, d = _dev(src), _dev(dst)
    want = tc.tc_count(s, d, n)
    assert _noalloc(tc, s, d, n) == (tc.TC_OK, want)  # warm-up: loads the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    tc.tc_debug_fail_allocations(0, 1 << 30)
    try:
        got = [_noalloc(tc, s, d, n) for _ in range(2)]
        # the ordinary entry point does allocate: it must fail meanwhile
        with pytest.raises(tc.TCError) as ei:
            tc.tc_count(s, d, n)
        assert ei.value.code == tc.TC_ERR_OOM
    finally:
        tc.tc_debug_fail_allocations(0, 0)
    torch.cuda.synchronize()
    assert got == [(tc.TC_OK, want)] * 2
    assert torch.cuda.mem_get_info()[0] == free0
