"""Pins for the CPU oracle: checks against facts fixed by mathematics.

The oracle restates the sequential forward algorithm (Sec. II-B).  Here it is
compared with things that do not depend on it: all-triples brute force,
trace(A^3)/6, sparse (A@A)*A, closed forms of named graph families,
invariants of the definition, and library routines.
"""
import math

import numpy as np
import pytest

import oracle
from graphgen import families as fam
from tests import helpers


def rand_simple(n, p, seed):
    return fam.gnp(n, p, seed)


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("n,p,seed", [(8, 0.5, 1), (16, 0.3, 2), (32, 0.25, 3), (48, 0.6, 4),
                                      (64, 0.1, 5), (64, 0.9, 6), (5, 1.0, 7), (1, 0.5, 8)])
def test_brute_force_simple(n, p, seed):
    s, d, n = rand_simple(n, p, seed)
    r = oracle.forward(s, d, n)
    T, t = helpers.brute_force(s, d, n)
    assert r["T"] == T
    assert np.array_equal(r["t"], t)


@pytest.mark.parametrize("n,m,seed", [(10, 60, 11), (24, 200, 12), (40, 500, 13), (64, 1500, 14)])
def test_brute_force_multigraph(n, m, seed):
    """Loops, repeats and both directions in the input collapse to one edge."""
    s, d, n = fam.random_multigraph(n, m, seed)
    r = oracle.forward(s, d, n)
    T, t = helpers.brute_force(s, d, n)
    assert r["T"] == T
    assert np.array_equal(r["t"], t)
    assert np.array_equal(r["deg"], helpers.simple_degrees(s, d, n))


# ------------------------------------------------------------------ algebra
@pytest.mark.parametrize("n,p,seed", [(200, 0.05, 21), (500, 0.02, 22), (1000, 0.01, 23),
                                      (300, 0.5, 24)])
def test_trace_a_cubed(n, p, seed):
    s, d, n = rand_simple(n, p, seed)
    r = oracle.forward(s, d, n)
    T, t = helpers.trace_cubed(s, d, n)
    assert r["T"] == T
    assert np.array_equal(r["t"], t)


def test_sparse_er16k():
    """The Erdos-Renyi workload (n=16384, m=131072) against scipy sparse."""
    import graphgen

    s, d, n = graphgen.workload("er16k")
    r = oracle.forward(s, d, n)
    T, t = helpers.sparse_counts(s, d, n)
    assert r["m"] == 131072
    assert r["T"] == T
    assert np.array_equal(r["t"], t)
    # E[T] = C(n,3) m(m-1)(m-2) / (N(N-1)(N-2)), N = C(n,2): about 683
    N = n * (n - 1) / 2
    expect = math.comb(n, 3) * 131072 * 131071 * 131070 / (N * (N - 1) * (N - 2))
    assert abs(T - expect) < 6 * math.sqrt(expect)


def test_sparse_rmat_power_law():
    """A skewed R-MAT graph (raw draws with repeats and loops)."""
    import graphgen

    s, d = graphgen.rmat(14, 16 << 14, 77)
    n = 1 << 14
    r = oracle.forward(s, d, n)
    T, t = helpers.sparse_counts(s, d, n)
    assert r["T"] == T and T > 0
    assert np.array_equal(r["t"], t)


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 10, 31, 64])
def test_complete(n):
    s, d, n = fam.complete(n)
    r = oracle.forward(s, d, n)
    assert r["T"] == math.comb(n, 3)
    assert np.all(r["t"] == math.comb(max(n - 1, 0), 2))


@pytest.mark.parametrize("builder", [
    lambda: fam.complete_bipartite(7, 9), lambda: fam.complete_bipartite(1, 30),
    lambda: fam.star(50), lambda: fam.path(40), lambda: fam.cycle(4), lambda: fam.cycle(17),
    lambda: fam.hypercube(6), lambda: fam.random_tree(300, 3), lambda: fam.grid(9, 13)])
def test_triangle_free(builder):
    s, d, n = builder()
    r = oracle.forward(s, d, n)
    assert r["T"] == 0
    assert not r["t"].any()


def test_triangle():
    r = oracle.forward([0, 1, 2], [1, 2, 0], 3)
    assert r["T"] == 1 and list(r["t"]) == [1, 1, 1]


@pytest.mark.parametrize("k", [3, 4, 5, 8, 100])
def test_wheel(k):
    """Rim of k vertices plus a hub: T = k for k >= 4; W with k=3 is K_4 (T=4)."""
    s, d, n = fam.wheel(k)
    r = oracle.forward(s, d, n)
    if k == 3:
        assert r["T"] == 4
    else:
        assert r["T"] == k
        assert r["t"][0] == k
        assert np.all(r["t"][1:] == 2)


@pytest.mark.parametrize("k", [1, 2, 7, 40])
def test_friendship(k):
    s, d, n = fam.friendship(k)
    r = oracle.forward(s, d, n)
    assert r["T"] == k
    assert r["t"][0] == k and np.all(r["t"][1:] == 1)


def test_disjoint_union_adds():
    g1, g2, g3 = fam.complete(9), fam.wheel(12), fam.friendship(5)
    s, d, n = fam.disjoint_union(g1, g2, g3)
    r = oracle.forward(s, d, n)
    assert r["T"] == math.comb(9, 3) + 12 + 5


def test_complete_with_tree():
    s, d, n = fam.complete_with_tree(20, 200, 5)
    r = oracle.forward(s, d, n)
    assert r["T"] == math.comb(20, 3)
    assert np.all(r["t"][20:] == 0)


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("seed", [31, 32, 33])
def test_sum_t_is_3T_and_relabel_invariance(seed):
    import graphgen

    s, d = graphgen.rmat(12, 16 << 12, seed)
    n = 1 << 12
    r = oracle.forward(s, d, n)
    assert int(r["t"].sum()) == 3 * r["T"]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int32)
    order = rng.permutation(len(s))
    flip = rng.random(len(s)) < 0.5
    s2, d2 = perm[s][order], perm[d][order]
    s3 = np.where(flip[order], d2, s2)
    d3 = np.where(flip[order], s2, d2)
    r2 = oracle.forward(s3, d3, n)
    assert r2["T"] == r["T"]
    assert np.array_equal(r2["t"][perm], r["t"])


def test_duplicates_and_loops_do_not_count():
    s, d, n = fam.gnp(150, 0.1, 41)
    base = oracle.forward(s, d, n)
    loops = np.arange(0, n, 3, dtype=np.int32)
    s2 = np.concatenate([s, d, s[:50], loops])
    d2 = np.concatenate([d, s, d[:50], loops])
    r = oracle.forward(s2, d2, n)
    assert r["T"] == base["T"] and r["m"] == base["m"]
    assert np.array_equal(r["t"], base["t"])


@pytest.mark.parametrize("seed", [51, 52])
def test_tie_break_direction_irrelevant(seed):
    import graphgen

    s, d = graphgen.rmat(11, 8 << 11, seed)
    n = 1 << 11
    a = oracle.forward(s, d, n)
    b = oracle.forward(s, d, n, tie_high_first=True)
    assert a["T"] == b["T"] and np.array_equal(a["t"], b["t"])


@pytest.mark.parametrize("builder", [
    lambda: fam.star(400), lambda: fam.complete(60), lambda: fam.wheel(300),
    lambda: fam.gnp(500, 0.05, 61)])
def test_forward_list_bound(builder):
    """max |N+(v)| <= floor(sqrt(2m)): every forward neighbour of v has
    degree >= deg(v) >= |N+(v)|, so |N+(v)|^2 <= sum of degrees = 2m; and the
    forward lists partition the edges, sum |N+(v)| = m."""
    s, d, n = builder()
    r = oracle.forward(s, d, n)
    od = oracle.out_degrees(s, d, n)
    assert int(od.sum()) == r["m"]
    assert r["max_out_degree"] == int(od.max()) if n else True
    assert r["max_out_degree"] <= math.isqrt(2 * r["m"])


def test_forward_list_bound_rmat():
    import graphgen

    s, d = graphgen.rmat(16, 16 << 16, 71)
    n = 1 << 16
    r = oracle.forward(s, d, n, per_vertex=False)
    assert r["max_out_degree"] <= math.isqrt(2 * r["m"])
    assert int(r["deg"].max()) > 20 * r["max_out_degree"]  # orientation tames the hubs


# ------------------------------------------------------------------ definition-based t(v)
@pytest.mark.parametrize("seed", [81, 82])
def test_vertex_triangles_matches_forward(seed):
    import graphgen

    s, d = graphgen.rmat(12, 16 << 12, seed)
    n = 1 << 12
    r = oracle.forward(s, d, n)
    vs = np.concatenate([np.argsort(-r["deg"])[:5], np.arange(0, n, 97)]).astype(np.int32)
    got = oracle.vertex_triangles(s, d, n, vs)
    assert np.array_equal(got, r["t"][vs])


def test_vertex_triangles_closed_forms():
    s, d, n = fam.wheel(9)
    assert list(oracle.vertex_triangles(s, d, n, [0, 1, 5])) == [9, 2, 2]
    s, d, n = fam.complete(12)
    assert list(oracle.vertex_triangles(s, d, n, [0, 11])) == [55, 55]


# ------------------------------------------------------------------ library routines
def test_networkx_triangles_clustering_transitivity():
    nx = pytest.importorskip("networkx")
    import graphgen

    s, d = graphgen.rmat(11, 12 << 11, 91)
    n = 1 << 11
    r = oracle.forward(s, d, n)
    g = nx.Graph()
    g.add_nodes_from(range(n))
    g.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
    tri = nx.triangles(g)
    assert np.array_equal(r["t"], np.array([tri[v] for v in range(n)], np.int64))
    cc = oracle.clustering(r["t"], r["deg"])
    ref = nx.clustering(g)
    assert np.allclose(cc, [ref[v] for v in range(n)], rtol=1e-15, atol=0)
    assert math.isclose(oracle.transitivity(r["T"], r["deg"]), nx.transitivity(g), rel_tol=1e-15)


def test_clustering_closed_forms():
    s, d, n = fam.complete(7)
    r = oracle.forward(s, d, n)
    assert np.all(oracle.clustering(r["t"], r["deg"]) == 1.0)
    assert oracle.transitivity(r["T"], r["deg"]) == 1.0
    s, d, n = fam.star(9)
    r = oracle.forward(s, d, n)
    assert np.all(oracle.clustering(r["t"], r["deg"]) == 0.0)
    assert oracle.transitivity(r["T"], r["deg"]) == 0.0
    s, d, n = fam.wheel(6)  # hub: 6 of C(6,2)=15 rim pairs; rim: 2 of C(3,2)=3
    r = oracle.forward(s, d, n)
    cc = oracle.clustering(r["t"], r["deg"])
    assert cc[0] == 6 / 15 and np.all(cc[1:] == 2 / 3)
    assert oracle.transitivity(0, np.zeros(4, np.int64)) == 0.0


# ------------------------------------------------------------------ errors
def test_errors():
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward([0, 5], [1, 2], 5)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward([0, -1], [1, 2], 5)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward([0], [1], -1)
    assert e.value.code in (1, 2)
    r = oracle.forward([], [], 0)
    assert r["T"] == 0 and r["m"] == 0
    r = oracle.forward([3, 3], [3, 3], 4)
    assert r["T"] == 0 and r["m"] == 0 and not r["deg"].any()
