"""Failure paths on the GPU, driven without faulting or hanging it.

* Bounded waits.  The preprocessing kernels wait on status words that
  earlier tiles publish (decoupled look-back); each wait gives up after a
  bounded number of iterations.  A test hook (include/tc_debug.h) makes one
  radix-sort tile never publish, so the tiles after it wait on a word that
  nothing sets until their (lowered) limit runs out.  The call must return
  TC_ERR_TIMEOUT -- no kernel may run on the incomplete data -- and the
  next call, with the defaults back, must count exactly.
* Allocation failures, injected on the host: the call returns TC_ERR_OOM,
  releases what it took, and the library stays usable.

The expected counts come from the CPU oracle.
"""
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
    yield lib
    lib.tc_debug_reset()


@pytest.fixture(scope="module")
def graph():
    """R-MAT scale 18 (4.2M pairs: about a thousand 4096-key radix tiles)."""
    src, dst = graphgen.rmat(18, 16 << 18, 31)
    n = 1 << 18
    return src, dst, n, oracle.forward(src, dst, n)


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def expect_error(tc, code, fn, *a, **k):
    with pytest.raises(tc.TCError) as ei:
        fn(*a, **k)
    assert ei.value.code == code, ei.value


@pytest.mark.parametrize("tile", [0, 3, 700])
def test_wait_on_unpublished_tile_times_out(tc, graph, tile):
    import torch

    src, dst, n, want = graph
    s, d = dev(src), dev(dst)
    tc.tc_debug_set_wait_limit(2000, tile)
    try:
        expect_error(tc, tc.TC_ERR_TIMEOUT, tc.tc_count, s, d, n)
        t = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        expect_error(tc, tc.TC_ERR_TIMEOUT, tc.tc_count_per_vertex, s, d, n, t_out=t)
        # nothing downstream ran: the per-vertex output was never written
        assert bool((t == -7).all().item())
    finally:
        tc.tc_debug_reset()
    torch.cuda.synchronize()  # the context is intact
    assert tc.tc_count(s, d, n) == want["T"]
    T, t, deg = tc.tc_count_per_vertex(s, d, n)
    assert T == want["T"] and np.array_equal(t.cpu().numpy(), want["t"])


def test_batch_and_engine_time_out_then_recover(tc, graph):
    src, dst, n, want = graph
    s, d = dev(np.concatenate([src, src])), dev(np.concatenate([dst, dst]))
    eo = np.array([0, len(src), 2 * len(src)], np.int64)
    vn = np.array([n, n], np.int32)
    tc.tc_debug_set_wait_limit(2000, 5)
    try:
        expect_error(tc, tc.TC_ERR_TIMEOUT, tc.tc_count_batch, s, d, eo, vn)
        with tc.Engine(2 * len(src), 2 * n, 4) as eng:
            expect_error(tc, tc.TC_ERR_TIMEOUT, eng.count, s, d, eo, vn)
            tc.tc_debug_reset()
            assert list(eng.count(s, d, eo, vn)) == [want["T"]] * 2
    finally:
        tc.tc_debug_reset()
    assert list(tc.tc_count_batch(s, d, eo, vn)) == [want["T"]] * 2


def test_tight_limit_never_gives_a_wrong_count(tc, graph):
    """With every wait limited to a single check, a call either counts
    exactly or reports the timeout: a wait that gives up never produces a
    number."""
    src, dst, n, want = graph
    s, d = dev(src), dev(dst)
    seen = set()
    tc.tc_debug_set_wait_limit(0, -1)
    try:
        for _ in range(4):
            try:
                got = tc.tc_count(s, d, n)
                assert got == want["T"]
                seen.add("ok")
            except tc.TCError as e:
                assert e.code == tc.TC_ERR_TIMEOUT, e
                seen.add("timeout")
    finally:
        tc.tc_debug_reset()
    assert seen
    assert tc.tc_count(s, d, n) == want["T"]


def test_allocation_failure_reports_oom_and_recovers(tc, graph):
    src, dst, n, want = graph
    s, d = dev(src), dev(dst)
    tc.tc_debug_fail_allocations(0, 1)
    expect_error(tc, tc.TC_ERR_OOM, tc.tc_count, s, d, n)
    assert tc.tc_count(s, d, n) == want["T"]
    # the host-buffer call takes several allocations: fail each in turn
    for skip in range(3):
        tc.tc_debug_fail_allocations(skip, 1)
        try:
            T, t, deg = tc.tc_count_per_vertex_host(src, dst, n)
            assert T == want["T"]  # fewer allocations than `skip` on this device
        except tc.TCError as e:
            assert e.code == tc.TC_ERR_OOM, e
        tc.tc_debug_fail_allocations(0, 0)
    T, t, deg = tc.tc_count_per_vertex_host(src, dst, n)
    assert T == want["T"] and np.array_equal(t, want["t"]) and np.array_equal(deg, want["deg"])
    tc.tc_debug_fail_allocations(0, 1)
    with pytest.raises(tc.TCError) as ei:
        tc.Engine(1 << 20, 1 << 16, 8)
    assert ei.value.code == tc.TC_ERR_OOM
    tc.tc_debug_fail_allocations(0, 0)
    with tc.Engine(len(src), n, 2) as eng:
        assert list(eng.count(s, d, np.array([0, len(src)], np.int64),
                              np.array([n], np.int32))) == [want["T"]]
