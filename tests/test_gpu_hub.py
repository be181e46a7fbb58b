"""The dense hub block (tensor-core count of the triangles among the 2^14
highest-ranked vertices) against the CPU oracle.

A single graph of at least 2^17 vertices counts the triangles whose lowest
vertex lies in the hub set H (the 2^14 vertices highest in the (degree, id)
order; the degree counts repeated input pairs, which changes the set but
never a count) as a masked 0/1 matrix product on the tensor cores, and leaves the
edges inside H out of the hash-set intersections.  The threshold
hub_min_edges (a tuning knob: counts never depend on it) forces the dense
block on (0) or off (-1), so the same graph is counted both ways; both must
equal the oracle exactly (integer counts: the tolerance is zero).
"""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import families as fam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1503_00576_gb300 as lib

    lib.load_library()
    yield lib
    lib.tc_set_tuning(None)


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def rmat17():
    src, dst = graphgen.rmat(17, 32 << 17, 51)
    return src, dst, 1 << 17


def clique_and_sparse():
    """K_200 beside a sparse random graph on 2^17 - 200 vertices: the clique's
    vertices have the highest degrees, so H holds it whole, plus the top of
    the sparse graph."""
    a = fam.complete(200)
    b_src, b_dst = graphgen.er((1 << 17) - 200, 600_000, 52)
    return fam.disjoint_union(a, (b_src, b_dst, (1 << 17) - 200))


@pytest.fixture(scope="module", params=["rmat17", "clique"])
def graph(request):
    src, dst, n = rmat17() if request.param == "rmat17" else clique_and_sparse()
    return src, dst, n, oracle.forward(src, dst, n)


@pytest.mark.parametrize("hub_min_edges", [0, -1])
def test_dense_and_hash_agree_with_the_oracle(tc, graph, hub_min_edges):
    src, dst, n, want = graph
    s, d = dev(src), dev(dst)
    tc.tc_set_tuning({"hub_min_edges": hub_min_edges})
    try:
        T, t, deg = tc.tc_count_per_vertex(s, d, n)
        assert T == want["T"]
        assert np.array_equal(t.cpu().numpy(), want["t"])
        assert np.array_equal(deg.cpu().numpy(), want["deg"])
        assert tc.tc_count(s, d, n) == want["T"]
    finally:
        tc.tc_set_tuning(None)


def test_dense_block_takes_the_hub_edges_off_the_hash_path(tc, graph):
    """With the dense block on, no lookup is left for an edge inside H (the
    2^14 highest ranks); with it off, those lookups are there, and the rest
    of the work is the same."""
    src, dst, n, want = graph
    s, d = dev(src), dev(dst)
    try:
        tc.tc_set_tuning({"hub_min_edges": 0})
        on = tc.tc_count_work(s, d, n)
        tc.tc_set_tuning({"hub_min_edges": -1})
        off = tc.tc_count_work(s, d, n)
    finally:
        tc.tc_set_tuning(None)
    h = 1 << 14
    assert on["hub_lookups"][h] == 0
    assert off["hub_lookups"][h] > 0
    assert off["lookups"] - on["lookups"] == off["hub_lookups"][h]
    assert on["triangles"] == off["triangles"] == want["T"]


def triangles_among_top_ranks(src, dst, n, H):
    """Triangles with all three vertices among the H vertices highest in the
    library's (degree, id) order -- the degree counting every non-loop input
    pair, repeats included -- : scipy on the induced subgraph."""
    import scipy.sparse as sp

    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    a, b = np.minimum(s, d)[keep], np.maximum(s, d)[keep]
    dord = np.bincount(a, minlength=n) + np.bincount(b, minlength=n)
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    top = np.zeros(n, bool)
    top[np.lexsort((np.arange(n), dord))[n - H:]] = True
    idx = np.full(n, -1, np.int64)
    idx[top] = np.arange(H)
    inside = top[a] & top[b]
    x, y = idx[a[inside]], idx[b[inside]]
    A = sp.coo_matrix((np.ones(len(x)), (x, y)), shape=(H, H)).tocsr()
    A = A + A.T
    return int(round((A @ A).multiply(A).sum())) // 6


def test_dense_triangles_match_the_top_ranks(tc, graph):
    """Forced on, the block covers the 2^14 highest-ranked vertices and
    counts exactly the triangles lying wholly among them."""
    src, dst, n, want = graph
    try:
        tc.tc_set_tuning({"hub_min_edges": 0})
        w = tc.tc_count_work(dev(src), dev(dst), n)
    finally:
        tc.tc_set_tuning(None)
    assert w["dense_vertices"] == 1 << 14
    assert w["dense_triangles"] == triangles_among_top_ranks(src, dst, n, 1 << 14)
    assert w["triangles"] == want["T"]


def test_cost_model_keeps_it_off_without_hubs(tc):
    """A random geometric graph of 2^17 vertices has no hubs: the estimated
    saving never pays for the product, so the block stays off."""
    n = 1 << 17
    src, dst = graphgen.rgg(n, graphgen.rgg_radius(n, 32.0), 54)
    w = tc.tc_count_work(dev(src), dev(dst), n)
    assert w["dense_vertices"] == 0 and w["dense_triangles"] == 0
    assert w["triangles"] == oracle.forward(src, dst, n, per_vertex=False)["T"]


def test_small_graphs_never_use_it(tc):
    """Below 2^17 vertices the layout has no hub block: forcing the knob
    changes nothing."""
    src, dst = graphgen.rmat(14, 32 << 14, 53)
    n = 1 << 14
    want = oracle.forward(src, dst, n)
    tc.tc_set_tuning({"hub_min_edges": 0})
    try:
        T, t, deg = tc.tc_count_per_vertex(dev(src), dev(dst), n)
    finally:
        tc.tc_set_tuning(None)
    assert T == want["T"] and np.array_equal(t.cpu().numpy(), want["t"])
    assert tc.tc_workspace_bytes(len(src), n) < tc.tc_workspace_bytes(len(src), 1 << 17)
