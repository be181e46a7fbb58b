"""GPU parity: libtc (through its C ABI) against the CPU oracle, bit-exact.

Counts are integers, so the tolerance is zero everywhere: T, t(v) and
deg(v) must be equal; the clustering coefficients and the transitivity ratio
are float64 results of the same expressions on the same integers, so they
must be equal too.
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
from graphgen import families as fam

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


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


def run_pv(tc, s, d, n):
    T, t, deg = tc.tc_count_per_vertex(dev(s), dev(d), n)
    return T, t.cpu().numpy(), deg.cpu().numpy()


def assert_same(tc, s, d, n, check_total_only=True):
    r = oracle.forward(s, d, n)
    T, t, deg = run_pv(tc, s, d, n)
    assert T == r["T"]
    assert np.array_equal(t, r["t"])
    assert np.array_equal(deg, r["deg"])
    if check_total_only:
        assert tc.tc_count(dev(s), dev(d), n) == r["T"]
    return r


# ------------------------------------------------------------------ small graphs
FAMILIES = {
    "triangle": lambda: (np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), 3),
    "K5": lambda: fam.complete(5),
    "K40": lambda: fam.complete(40),
    "K300": lambda: fam.complete(300),
    "wheel5": lambda: fam.wheel(5),
    "wheel1000": lambda: fam.wheel(1000),
    "friendship50": lambda: fam.friendship(50),
    "star2000": lambda: fam.star(2000),
    "bipartite": lambda: fam.complete_bipartite(20, 70),
    "hypercube8": lambda: fam.hypercube(8),
    "grid": lambda: fam.grid(40, 50),
    "tree": lambda: fam.random_tree(5000, 1),
    "union": lambda: fam.disjoint_union(fam.complete(30), fam.wheel(77), fam.friendship(9)),
    "clique_tree": lambda: fam.complete_with_tree(120, 3000, 4),
}


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_families(tc, name):
    s, d, n = FAMILIES[name]()
    assert_same(tc, s, d, n)


@pytest.mark.parametrize("n,p,seed", [(30, 0.5, 1), (200, 0.1, 2), (1000, 0.02, 3),
                                      (3000, 0.01, 4), (500, 0.6, 5)])
def test_gnp(tc, n, p, seed):
    s, d, n = fam.gnp(n, p, seed)
    assert_same(tc, s, d, n)


@pytest.mark.parametrize("n,m,seed", [(5, 40, 1), (50, 3000, 2), (4000, 60000, 3),
                                      (100000, 400000, 4)])
def test_multigraph_input(tc, n, m, seed):
    """Loops, repeats and reversed copies in the input."""
    s, d, n = fam.random_multigraph(n, m, seed)
    assert_same(tc, s, d, n)


@pytest.mark.parametrize("scale,ef,seed", [(8, 8, 11), (12, 16, 12), (16, 16, 13),
                                           (18, 8, 14)])
def test_rmat(tc, scale, ef, seed):
    import graphgen

    s, d = graphgen.rmat(scale, ef << scale, seed)
    assert_same(tc, s, d, 1 << scale)


def test_rgg_small(tc):
    import graphgen

    n = 100000
    s, d = graphgen.rgg(n, graphgen.rgg_radius(n), 21)
    assert_same(tc, s, d, n)


# ------------------------------------------------------------------ edge cases
def test_empty(tc):
    e = np.zeros(0, np.int32)
    assert tc.tc_count(dev(e), dev(e), 10) == 0
    T, t, deg = run_pv(tc, e, e, 10)
    assert T == 0 and not t.any() and not deg.any()
    assert tc.tc_count(dev(e), dev(e), 0) == 0


def test_single_vertex_and_loops(tc):
    s = np.zeros(100, np.int32)
    assert tc.tc_count(dev(s), dev(s), 1) == 0
    s = np.arange(50, dtype=np.int32)
    T, t, deg = run_pv(tc, s, s, 50)
    assert T == 0 and not deg.any()


def test_all_duplicates(tc):
    s = np.array([0, 1, 2] * 1000 + [1, 2, 0] * 1000, np.int32)
    d = np.array([1, 2, 0] * 1000 + [0, 1, 2] * 1000, np.int32)
    T, t, deg = run_pv(tc, s, d, 3)
    assert T == 1 and list(t) == [1, 1, 1] and list(deg) == [2, 2, 2]


def test_paper_format_each_edge_twice(tc):
    """Sec. III-A lists every edge in both directions; the count is the same."""
    import graphgen

    s, d = graphgen.er(5000, 40000, 31)
    once = tc.tc_count(dev(s), dev(d), 5000)
    twice = tc.tc_count(dev(np.concatenate([s, d])), dev(np.concatenate([d, s])), 5000)
    assert once == twice == oracle.forward(s, d, 5000)["T"]


@pytest.mark.parametrize("k", [200, 300, 600, 3000, 8200])
def test_repeated_edges_in_long_lists(tc, k):
    """K_k with every edge given in both directions and a third of them a
    third time, in shuffled order: each forward list holds every entry two
    or three times before the list sort drops the repeats.  The lists of
    up to 2k entries take the warp sort (k = 200), the warp sort of up to
    1024 keys (300), the CTA sort in shared memory (600, 3000) and the
    chunked sort merged in global memory (8200: lists of up to 24597
    entries).  T = C(k,3), t(v) = C(k-1,2), deg(v) = k-1."""
    a, b = (x.astype(np.int32) for x in np.triu_indices(k, 1))
    rng = np.random.default_rng(k)
    third = rng.random(len(a)) < 1 / 3
    s = np.concatenate([a, b, a[third]])
    d = np.concatenate([b, a, b[third]])
    order = rng.permutation(len(s))
    s, d = s[order], d[order]
    T, t, deg = run_pv(tc, s, d, k)
    assert T == math.comb(k, 3)
    assert np.all(t == math.comb(k - 1, 2)) and np.all(deg == k - 1)
    assert tc.tc_count(dev(s), dev(d), k) == T


def test_id_out_of_range(tc):
    s = np.array([0, 1, 5], np.int32)
    d = np.array([1, 2, 0], np.int32)
    with pytest.raises(tc.TCError) as e:
        tc.tc_count(dev(s), dev(d), 5)
    assert e.value.code == tc.TC_ERR_ID_RANGE
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_per_vertex(dev(np.array([0, -3], np.int32)), dev(np.array([1, 2], np.int32)), 5)
    assert e.value.code == tc.TC_ERR_ID_RANGE
    with pytest.raises(tc.TCError) as e:
        tc.tc_count(dev(s), dev(d), 0)
    assert e.value.code == tc.TC_ERR_ID_RANGE
    # the library stays usable after an error
    assert tc.tc_count(dev(d), dev(s[::-1].copy()), 6) >= 0


def test_invalid_arguments(tc):
    lib = tc.load_library()
    assert lib.tc_count(None, None, -1, 5, None) == tc.TC_COUNT_ERROR
    assert lib.tc_last_error() == tc.TC_ERR_INVALID_ARG
    assert lib.tc_count(None, None, 1 << 31, 5, None) == tc.TC_COUNT_ERROR
    assert lib.tc_last_error() == tc.TC_ERR_OVERFLOW
    assert lib.tc_count(None, None, 3, 5, None) == tc.TC_COUNT_ERROR
    assert lib.tc_last_error() == tc.TC_ERR_INVALID_ARG


@pytest.mark.parametrize("row", [0, 1, 2, 7, 8, 9, 15, 16, 17, 31, 32, 33, 64, 127, 128, 129,
                                 255, 256, 257, 1000, 1024, 1025])
def test_row_lengths(tc, row):
    """A vertex whose forward list has exactly `row` entries: a clique on
    row+1 vertices (equal degrees, so the lowest id owns the longest list)
    plus a path and a star that add no triangle.  The lengths straddle the
    32-byte blocks the lists are padded to (8 entries), the warp-group limit
    (128) and the CTA-group limit (1024, past which the long-list kernel
    takes the group)."""
    s, d, n = fam.disjoint_union(fam.complete(row + 1), fam.path(50), fam.star(40))
    r = assert_same(tc, s, d, n, check_total_only=False)
    assert r["max_out_degree"] == max(row, 1)


@pytest.mark.parametrize("row", [4096, 4097, 5000])
def test_long_rows_closed_form(tc, row):
    """Rows of 4096 entries fill half the long-list kernel's table; longer
    ones are hashed in two segments.  A clique on k vertices has C(k,3)
    triangles and C(k-1,2) at every vertex."""
    k = row + 1
    s, d, n = fam.disjoint_union(fam.complete(k), fam.path(50), fam.star(40))
    T, t, deg = run_pv(tc, s, d, n)
    assert T == math.comb(k, 3)
    assert np.all(t[:k] == math.comb(k - 1, 2)) and not t[k:].any()
    assert np.all(deg[:k] == k - 1)


def test_long_row_global_fallback(tc):
    """K_8200: the lowest ids own forward lists longer than 8192 entries,
    hashed in three segments, each probed by every partner.  T = C(n,3)
    exactly."""
    n = 8200
    s, d, n = fam.complete(n)
    T, t, deg = run_pv(tc, s, d, n)
    assert T == math.comb(n, 3)
    assert np.all(t == math.comb(n - 1, 2)) and np.all(deg == n - 1)


def test_relabel_invariance(tc):
    import graphgen

    s, d = graphgen.rmat(16, 16 << 16, 41)
    n = 1 << 16
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    a = tc.tc_count(dev(s), dev(d), n)
    b = tc.tc_count(dev(perm[d]), dev(perm[s]), n)
    assert a == b == oracle.forward(s, d, n, per_vertex=False)["T"]


def spread(s, d, n_small, n, seed):
    """The graph (s, d) on [0, n_small) with its ids sent to distinct random
    ids of [0, n), n - 1 among them; every other id of [0, n) is isolated."""
    rng = np.random.default_rng(seed)
    ids = np.empty(n_small, np.int64)
    ids[:-1] = rng.choice(n - 1, size=n_small - 1, replace=False)
    ids[-1] = n - 1
    ids = ids[rng.permutation(n_small)].astype(np.int32)
    return ids[s], ids[d]


@pytest.mark.parametrize("n", [1 << 24, (1 << 24) + 1, (1 << 26) + 777])
def test_wide_id_ranges(tc, n):
    """Ids of 24, 25 and 27 bits: past 24 bits the keys leave no room for the
    skipped blocks (every list is streamed whole), the dense hub block is off,
    and every sort takes a fourth radix pass; 2^24 and 2^24 + 1 hold the same
    edges on either side of that line (the extra vertex is isolated)."""
    import graphgen

    s, d = graphgen.rmat(17, 24 << 17, 47)
    S, D = spread(s, d, 1 << 17, n, 9)
    r = assert_same(tc, S, D, n)
    assert r["T"] == oracle.forward(s, d, 1 << 17, per_vertex=False)["T"]


@pytest.mark.parametrize("n,k", [(1000, 5), (300_001, 25)])
def test_ring_lattice_closed_form(tc, n, k):
    """The Watts-Strogatz lattice before rewiring: n C(k, 2) triangles, 3 C(k, 2)
    at every vertex, every degree 2k (all degrees equal: the order is the
    permuted ids alone)."""
    import graphgen

    s, d = graphgen.ws(n, k, 0.0, 12)
    T, t, deg = run_pv(tc, s, d, n)
    assert T == n * math.comb(k, 2) == tc.tc_count(dev(s), dev(d), n)
    assert np.all(t == 3 * math.comb(k, 2)) and np.all(deg == 2 * k)


def test_clustering_and_transitivity(tc):
    import graphgen

    s, d = graphgen.rmat(14, 16 << 14, 51)
    n = 1 << 14
    r = oracle.forward(s, d, n)
    T, t, deg = tc.tc_count_per_vertex(dev(s), dev(d), n)
    cc, tr = tc.tc_clustering(t, deg)
    assert np.array_equal(cc.cpu().numpy(), oracle.clustering(r["t"], r["deg"]))
    assert tr == oracle.transitivity(r["T"], r["deg"])
    s, d, n = fam.complete(9)
    T, t, deg = tc.tc_count_per_vertex(dev(s), dev(d), n)
    cc, tr = tc.tc_clustering(t, deg)
    assert tr == 1.0 and bool((cc == 1.0).all())


def test_host_buffers(tc):
    import graphgen

    s, d = graphgen.rmat(15, 16 << 15, 61)
    n = 1 << 15
    r = oracle.forward(s, d, n)
    assert tc.tc_count_host(s, d, n) == r["T"]
    T, t, deg = tc.tc_count_per_vertex_host(s, d, n)
    assert T == r["T"] and np.array_equal(t, r["t"]) and np.array_equal(deg, r["deg"])


def test_host_buffers_pinned_and_bad_ids(tc):
    """Page-locked inputs and outputs (the bench's end-to-end call), a ragged
    pair count, and an id out of range reported through the host call."""
    import torch
    import graphgen

    s, d = graphgen.rmat(16, (16 << 16) + 13, 62)
    n = 1 << 16
    r = oracle.forward(s, d, n)
    hs, hd = torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory()
    ht = torch.empty(n, dtype=torch.int64).pin_memory()
    hdeg = torch.empty(n, dtype=torch.int32).pin_memory()
    assert tc.tc_count_host(hs, hd, n) == r["T"]
    T, _, _ = tc.tc_count_per_vertex_host(hs, hd, n, t_out=ht, deg_out=hdeg)
    assert T == r["T"]
    assert np.array_equal(ht.numpy(), r["t"]) and np.array_equal(hdeg.numpy(), r["deg"])
    bad = d.copy()
    bad[len(bad) // 2] = n
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_host(s, bad, n)
    assert e.value.code == tc.TC_ERR_ID_RANGE


def test_caller_workspace(tc):
    import torch
    import graphgen

    s, d = graphgen.rmat(15, 16 << 15, 71)
    n = 1 << 15
    need = tc.tc_workspace_bytes(len(s), n)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    want = oracle.forward(s, d, n, per_vertex=False)["T"]
    assert tc.tc_count_ws(dev(s), dev(d), n, ws) == want
    assert tc.tc_count_ws(dev(s), dev(d), n, ws) == want  # reusable
    with pytest.raises(tc.TCError) as e:
        tc.tc_count_ws(dev(s), dev(d), n, ws[: need // 2])
    assert e.value.code == tc.TC_ERR_INVALID_ARG


def test_side_stream_and_repeat(tc):
    import torch
    import graphgen

    s, d = graphgen.rmat(17, 16 << 17, 81)
    n = 1 << 17
    want = oracle.forward(s, d, n, per_vertex=False)["T"]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ds, dd = dev(s), dev(d)
        got = [tc.tc_count(ds, dd, n, stream=st) for _ in range(3)]
    assert got == [want] * 3


def test_launch_counter_and_profile(tc):
    import graphgen

    s, d = graphgen.rmat(12, 16 << 12, 91)
    before = tc.tc_launch_count()
    tc.tc_profile_enable(True)
    tc.tc_profile_read(reset=True)
    tc.tc_count(dev(s), dev(d), 1 << 12)
    prof = tc.tc_profile_read(reset=True)
    tc.tc_profile_enable(False)
    launched = tc.tc_launch_count() - before
    assert launched >= 8
    assert sum(x[1] for x in prof.values()) == launched
    # the count phase (total only) launches the long-list kernel and the
    # main kernel
    assert all(ms >= 0.0 for ms, _ in prof.values()) and prof["count"][1] == 2


# ------------------------------------------------------------------ full-size workloads
def _golden(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]


def _input(name):
    import graphgen

    g = _golden(name)
    s, d, n = graphgen.workload(name)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s, "<i4").tobytes())
    h.update(np.ascontiguousarray(d, "<i4").tobytes())
    assert h.hexdigest() == g["input_sha256"], "generator output differs on this host"
    return s, d, n, g


def test_er16k_full(tc):
    s, d, n, g = _input("er16k")
    r = assert_same(tc, s, d, n)
    assert r["T"] == g["T"]


@pytest.mark.parametrize("name", ["rmat20", "rgg4m", "rmat24", "ba200k", "ws1m"])
def test_workload_full(tc, name):
    """Full-size workloads against the oracle's stored results: T, the SHA-256
    of all per-vertex counts and degrees, sampled t(v), sum t = 3T."""
    import torch

    s, d, n, g = _input(name)
    ds, dd = dev(s), dev(d)
    T, t, deg = tc.tc_count_per_vertex(ds, dd, n)
    assert T == g["T"]
    assert tc.tc_count(ds, dd, n) == g["T"]
    th = t.cpu().numpy()
    dh = deg.cpu().numpy()
    vs = np.array(g["sample_vertices"], np.int64)
    assert th[vs].tolist() == g["sample_t"]
    assert dh[vs].tolist() == g["sample_deg"]
    assert int(th.sum()) == 3 * g["T"]
    assert hashlib.sha256(np.ascontiguousarray(th, "<i8").tobytes()).hexdigest() == g["t_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(dh, "<i4").tobytes()).hexdigest() == g["deg_sha256"]
    _, tr = tc.tc_clustering(t, deg, want_cc=False)
    assert tr == g["transitivity"]
    del ds, dd, t, deg
    torch.cuda.empty_cache()
