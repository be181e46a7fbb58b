"""Shares of the counting work (the multi-GPU setup of Sec. III-E), run one
after another on one GPU: the shares of parts 0 .. P-1 must add up exactly
to the whole count (T and every t(v)), every share must carry a like part
of the work, and the degrees must be complete in every share.  Counts are
integers: the tolerance is zero.  Each share is a separate call, so this
also checks that the dealing of groups to shares does not depend on the
order in which one call happens to bin them."""
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


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


@pytest.fixture(scope="module")
def rmat16():
    src, dst = graphgen.rmat(16, 16 << 16, 21)
    return dev(src), dev(dst), 1 << 16


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_total_shares_add_up(tc, rmat16, parts):
    s, d, n = rmat16
    whole = tc.tc_count(s, d, n)
    shares = [tc.tc_count_part(s, d, n, p, parts) for p in range(parts)]
    assert sum(shares) == whole
    if 1 < parts <= 3:  # consecutive degree ranks alternate: like shares
        assert min(shares) > 0.6 * whole / parts
        assert max(shares) < 1.4 * whole / parts


@pytest.mark.parametrize("parts", [2, 3, 8])
def test_shares_carry_like_work(tc, rmat16, parts):
    """Every share's counting work (hash lookups of its partner groups,
    tc_count_work_part) is within 10% of an equal split, and the shares'
    work adds up to the whole graph's."""
    s, d, n = rmat16
    whole = tc.tc_count_work(s, d, n)
    shares = [tc.tc_count_work(s, d, n, part=p, parts=parts) for p in range(parts)]
    for key in ("lookups", "inserts", "merge_work", "triangles"):
        assert sum(w[key] for w in shares) == whole[key], key
    mean = whole["lookups"] / parts
    for w in shares:
        assert 0.9 * mean < w["lookups"] < 1.1 * mean, [x["lookups"] for x in shares]


def test_per_vertex_shares_add_up_to_the_oracle(tc):
    src, dst = graphgen.rmat(12, 16 << 12, 22)
    n = 1 << 12
    want = oracle.forward(src, dst, n)
    s, d = dev(src), dev(dst)
    acc = np.zeros(n, np.int64)
    total = 0
    for p in range(3):
        T, t, deg = tc.tc_count_per_vertex_part(s, d, n, p, 3)
        total += T
        acc += t.cpu().numpy()
        assert np.array_equal(deg.cpu().numpy(), want["deg"])
    assert total == want["T"]
    assert np.array_equal(acc, want["t"])


@pytest.mark.parametrize("parts", [2, 3])
def test_shares_add_up_with_the_dense_hub_block(tc, parts):
    """A graph of 2^17 vertices with the dense hub block forced on: the
    block is counted by part 0 alone and every part leaves its edges off
    the hash path, so the shares of T and of every t(v) still add up to the
    oracle's."""
    src, dst = graphgen.rmat(17, 32 << 17, 24)
    n = 1 << 17
    want = oracle.forward(src, dst, n)
    s, d = dev(src), dev(dst)
    tc.tc_set_tuning({"hub_min_edges": 0})
    try:
        assert sum(tc.tc_count_part(s, d, n, p, parts) for p in range(parts)) == want["T"]
        acc = np.zeros(n, np.int64)
        total = 0
        for p in range(parts):
            T, t, deg = tc.tc_count_per_vertex_part(s, d, n, p, parts)
            total += T
            acc += t.cpu().numpy()
        assert total == want["T"] and np.array_equal(acc, want["t"])
    finally:
        tc.tc_set_tuning(None)


def test_shares_of_a_batchless_empty_graph(tc):
    import torch

    e = torch.empty(0, dtype=torch.int32, device="cuda")
    assert [tc.tc_count_part(e, e, 10, p, 2) for p in range(2)] == [0, 0]


@pytest.mark.parametrize("part,parts", [(0, 0), (-1, 2), (2, 2), (5, 3)])
def test_bad_shares_are_rejected(tc, rmat16, part, parts):
    s, d, n = rmat16
    with pytest.raises(tc.TCError) as err:
        tc.tc_count_part(s, d, n, part, parts)
    assert err.value.code == tc.TC_ERR_INVALID_ARG
