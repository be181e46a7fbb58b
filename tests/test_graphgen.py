"""The seeded input generators: determinism and the family definitions."""
import hashlib
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


def _canon(s, d):
    a = np.minimum(s, d).astype(np.int64)
    b = np.maximum(s, d).astype(np.int64)
    return a << 32 | b


def test_er_exact_m_no_loops():
    s, d = graphgen.er(1000, 20000, 5)
    assert len(s) == 20000
    assert np.all(s != d)
    assert len(np.unique(_canon(s, d))) == 20000
    assert s.min() >= 0 and max(s.max(), d.max()) < 1000


def test_er_complete_limit():
    s, d = graphgen.er(20, 190, 9)
    assert len(np.unique(_canon(s, d))) == 190
    with pytest.raises(ValueError):
        graphgen.er(20, 191, 9)


def test_rmat_range_and_skew():
    s, d = graphgen.rmat(12, 1 << 16, 3, permute=False)
    assert s.min() >= 0 and max(s.max(), d.max()) < 4096
    deg = np.bincount(np.concatenate([s, d]), minlength=4096)
    # with a = 0.57 the all-zero-bits vertex is the heaviest
    assert deg[0] == deg.max()


def test_rmat_distinct():
    s, d = graphgen.rmat_distinct(13, 50000, 4)
    assert len(s) == 50000
    assert np.all(s != d)
    assert len(np.unique(_canon(s, d))) == 50000
    raw_s, raw_d = graphgen.rmat(13, 60000, 4)
    keep = raw_s != raw_d
    # the output is the first-occurrence subsequence of the raw draw stream
    key = _canon(raw_s[keep], raw_d[keep])
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)[:50000]
    assert np.array_equal(s, raw_s[keep][first]) and np.array_equal(d, raw_d[keep][first])


def test_rgg_distance_rule():
    n, seed = 3000, 11
    r = graphgen.rgg_radius(n, 20.0)
    s, d = graphgen.rgg(n, r, seed)
    x, y, perm = graphgen.rgg_points(n, seed)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    # brute force over all pairs, same float64 expression
    dx = x[:, None] - x[None, :]
    dy = y[:, None] - y[None, :]
    close = (dx * dx + dy * dy) < r * r
    iu = np.triu_indices(n, 1)
    sel = close[iu]
    want = np.sort(_canon(perm[iu[0][sel]], perm[iu[1][sel]]))
    got = np.sort(_canon(s, d))
    assert np.array_equal(got, want)
    assert len(np.unique(got)) == len(got)


@pytest.mark.parametrize("threads", ["1", "3"])
def test_thread_count_independent(threads):
    code = ("import hashlib, graphgen as g\n"
            "h = hashlib.sha256()\n"
            "for a in (g.rmat(14, 300000, 5), g.rmat_distinct(14, 100000, 6), "
            "g.rgg(20000, g.rgg_radius(20000), 7), g.ws(20000, 5, 0.3, 8)):\n"
            "    h.update(a[0].tobytes()); h.update(a[1].tobytes())\n"
            "print(h.hexdigest())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in (threads, "8"):
        env = dict(os.environ, GG_THREADS=t)
        outs.append(subprocess.check_output([sys.executable, "-c", code], cwd=root, env=env))
    assert outs[0] == outs[1]


@pytest.mark.parametrize("name", ["er16k", "rmat20", "rgg4m", "ba200k", "ws1m"])
def test_workload_hash_matches_golden(name):
    """The stored input hashes pin the generator across hosts."""
    with open(GOLDEN) as f:
        gold = json.load(f)[name]
    s, d, n = graphgen.workload(name)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s, "<i4").tobytes())
    h.update(np.ascontiguousarray(d, "<i4").tobytes())
    assert h.hexdigest() == gold["input_sha256"]
    assert n == gold["n"] and len(s) == gold["m_in"]


def test_rgg_mean_degree():
    n = 200000
    s, d = graphgen.rgg(n, graphgen.rgg_radius(n), 3)
    mean = 2 * len(s) / n
    assert 31.0 < mean < 32.0  # boundary effects lower it slightly below 32


def test_graph_batch_deterministic_and_simple():
    a = graphgen.graph_batch(24, 3, log2_n=(6, 11))
    b = graphgen.graph_batch(24, 3, log2_n=(6, 11), threads=1)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert np.array_equal(a.edge_offsets, b.edge_offsets)
    n, m, kinds, _ = graphgen.batch_params(24, 3, log2_n=(6, 11))
    assert np.array_equal(np.diff(a.edge_offsets), m)
    assert kinds[0] == "er" and kinds[1] == "rmat"
    for g in range(len(a)):
        s, d, nv = a.graph(g)
        assert nv == n[g] and len(s) == m[g]
        assert np.all(s != d) and s.min(initial=0) >= 0 and max(s.max(initial=0), d.max(initial=0)) < nv
        assert len(np.unique(_canon(s, d))) == len(s)


def test_batch_params_ranges():
    n, m, kinds, _ = graphgen.batch_params(4096, 1005)
    assert n.min() >= 256 and n.max() <= 1 << 18
    d = 2 * m / n
    assert d.min() >= 3.9 and d.max() <= 64.0
    assert kinds.count("er") == kinds.count("rmat") == 2048


# ------------------------------------------------------------ Barabasi-Albert
def test_ba_structure():
    n, k = 3000, 7
    s, d = graphgen.ba(n, k, 21)
    assert len(s) == k * (k + 1) // 2 + (n - k - 1) * k
    assert np.all(s != d)
    assert len(np.unique(_canon(s, d))) == len(s)  # picks of a vertex are distinct
    assert s.min() >= 0 and max(s.max(), d.max()) < n
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert deg.min() >= k
    # preferential attachment: a few early vertices collect far more than k
    assert deg.max() > 6 * k
    s2, d2 = graphgen.ba(n, k, 21)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_ba_first_vertices_closed_form(k):
    """n = k + 1 is the seed clique; one more vertex joins k of its k + 1
    vertices and closes C(k, 2) more triangles."""
    import oracle

    s, d = graphgen.ba(k + 1, k, 3)
    assert oracle.forward(s, d, k + 1, per_vertex=False)["T"] == math.comb(k + 1, 3)
    s, d = graphgen.ba(k + 2, k, 3)
    assert oracle.forward(s, d, k + 2, per_vertex=False)["T"] == math.comb(k + 1, 3) + math.comb(k, 2)


# ------------------------------------------------------------ Watts-Strogatz
@pytest.mark.parametrize("n,k", [(16, 5), (1000, 5), (4001, 13)])
def test_ws_lattice_closed_form(n, k):
    """p = 0 leaves the ring lattice: with n >= 3k + 1 each triangle lies
    within k + 1 consecutive vertices, n C(k, 2) of them, 3 C(k, 2) at each
    vertex, every degree 2k."""
    import oracle

    s, d = graphgen.ws(n, k, 0.0, 5)
    assert len(s) == n * k and len(np.unique(_canon(s, d))) == n * k
    r = oracle.forward(s, d, n)
    assert r["T"] == n * math.comb(k, 2)
    assert np.all(r["t"] == 3 * math.comb(k, 2)) and np.all(r["deg"] == 2 * k)


def test_ws_rewiring():
    import oracle

    n, k = 20000, 10
    s, d = graphgen.ws(n, k, 0.1, 6)
    assert len(s) == n * k and np.all(s != d)
    r = oracle.forward(s, d, n)
    # clustering of the lattice, 3(k-1) / (2(2k-1)), thinned by (1-p)^3
    want = 3 * (k - 1) / (2 * (2 * k - 1)) * 0.9 ** 3
    assert abs(oracle.transitivity(r["T"], r["deg"]) - want) < 0.02
    # every edge moved: a sparse random graph keeps few triangles
    s, d = graphgen.ws(n, k, 1.0, 6)
    assert oracle.forward(s, d, n, per_vertex=False)["T"] < 3000
    with pytest.raises(ValueError):
        graphgen.ws(2 * k + 1, k, 0.1, 6)


def test_graph_batch_subset_equals_the_whole():
    full = graphgen.graph_batch(64, 77, log2_n=(6, 12))
    pick = [5, 0, 63, 17]
    sub = graphgen.graph_batch(64, 77, log2_n=(6, 12), only=pick)
    assert len(sub) == len(pick)
    for j, g in enumerate(pick):
        a, b, n = sub.graph(j)
        x, y, m = full.graph(g)
        assert n == m and np.array_equal(a, x) and np.array_equal(b, y)
        assert sub.kinds[j] == full.kinds[g] and sub.seeds[j] == full.seeds[g]
