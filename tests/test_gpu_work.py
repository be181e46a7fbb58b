"""Work counters of the counting phase (tc_count_work) against numpy.

The library orders the vertices by (degree counted with repeated input
pairs, id): without repeats that is the order of Sec. II-B, and any order
gives the same counts.  From that order and the cleaned edge set numpy
gives every forward-list length d+(v) and the expected work follows:
lookups = sum over edges of the streamed (shorter, ties to the non-owner)
list less its skipped leading blocks, inserts = the hashed lists of the
partner groups, W = sum over edges of d+(u) + d+(v) = sum over v of
deg(v) d+(v), max d+ <= sqrt(2m).

Skipped blocks: forward lists are sorted (by (degree, id) rank).  When the
edge's non-owner v has the longer list (h = v), the owner's list N+(u) is
streamed, and its entries before v's own place in it are below v, so not
in N+(v): the whole 8-entry blocks among them are skipped.
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
    return lib


def expected_work(src, dst, n):
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    a, b = np.minimum(s, d)[keep], np.maximum(s, d)[keep]
    # the order's degree counts every non-loop pair, repeats included
    dord = np.bincount(a, minlength=n) + np.bincount(b, minlength=n)
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    deg = np.bincount(a, minlength=n) + np.bincount(b, minlength=n)
    # owner = the endpoint lower in the (degree with repeats, id) order
    a_first = (dord[a] < dord[b]) | ((dord[a] == dord[b]) & (a < b))
    u = np.where(a_first, a, b)
    v = np.where(a_first, b, a)
    dp = np.bincount(u, minlength=n).astype(np.int64)
    if not (dord > deg).any():  # no repeats: the oracle's orientation
        assert np.array_equal(dp, oracle.out_degrees(src, dst, n))
    du, dv = dp[u], dp[v]
    h = np.where(dv > du, v, u)  # the longer list is hashed; ties stay at the owner
    l = np.where(dv > du, u, v)
    lookups_full = np.minimum(du, dv).sum()
    inserts = dp[np.unique(h)].sum()
    W = (du + dv).sum()
    assert W == (deg * dp).sum()  # the two forms of the merge work agree
    assert dp.sum() == len(key)
    # hub sets: the 2^12 .. 2^15 vertices highest in the order
    order = np.lexsort((np.arange(n), dord))  # ascending degree, then id
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    # sorted forward lists in rank space: N+(u) holds the ranks of u's
    # forward neighbours, ascending; pos = the place of v in N+(u)
    ru, rv = rank[u], rank[v]
    comp = ru * (n + 1) + rv
    pos = np.searchsorted(np.sort(comp), comp) - np.searchsorted(np.sort(comp), ru * (n + 1))
    # h = v: N+(u) is streamed and its entries before v (all below v, so not
    # in N+(v)) fill pos >> 3 whole blocks that are skipped
    skip = np.where(dv > du, pos >> 3, 0)
    streamed = np.where(dv > du, du, dv) - 8 * skip
    lookups = streamed.sum()
    assert lookups <= lookups_full
    hub = {}
    for k in range(4):
        size = 1 << (12 + k)
        inside = (rank[u] >= n - size) & (rank[v] >= n - size)
        hub[size] = int(streamed[inside].sum())
    return {"edges": len(key), "lookups": int(lookups), "inserts": int(inserts),
            "merge_work": int(W), "max_out_degree": int(dp.max()) if n else 0,
            "hub_lookups": hub, "dense_vertices": 0, "dense_triangles": 0}


@pytest.mark.parametrize("case", ["rmat12", "er", "k9", "rgg", "rmat16"])
def test_work_matches_oracle(tc, case):
    import torch

    if case == "rmat12":
        src, dst = graphgen.rmat(12, 16 << 12, 9)
        n = 1 << 12
    elif case == "er":
        src, dst = graphgen.er(3000, 20000, 4)
        n = 3000
    elif case == "k9":
        src, dst = (np.asarray(x, np.int32) for x in np.triu_indices(9, 1))
        n = 9
    elif case == "rgg":
        src, dst = graphgen.rgg(1 << 13, graphgen.rgg_radius(1 << 13, 12.0), 6)
        n = 1 << 13
    else:  # more vertices than the largest hub set
        src, dst = graphgen.rmat(16, 16 << 16, 10)
        n = 1 << 16
    want = expected_work(src, dst, n)
    want["triangles"] = oracle.forward(src, dst, n, per_vertex=False)["T"]
    want["vertices"] = n
    got = tc.tc_count_work(torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda(), n)
    assert got == want
    assert got["max_out_degree"] ** 2 <= 2 * got["edges"]
    # nested hub sets: shares grow with |H| and reach all lookups once |H| >= n
    hub = [got["hub_lookups"][1 << (12 + k)] for k in range(4)]
    assert hub == sorted(hub) and hub[-1] <= got["lookups"]
    if n <= 1 << 12:
        assert hub == [got["lookups"]] * 4
    if case == "k9":  # K_n: d+ = n-1, ..., 0, so W = (n-1) C(n,2) and lookups = C(n,3)
        assert got["merge_work"] == 8 * 36 and got["lookups"] == 84 == got["triangles"]
